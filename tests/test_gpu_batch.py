"""GPU parity of the persistent batched kernel (sv_batch_*) against the CPU oracle, and the
batching identity: an instance's result is bit-identical alone and inside any batch."""
import numpy as np
import pytest

import oracle
from paper_2601_09951_gb300 import svqe
from paper_2601_09951_gb300 import workloads as W
from tests.parity import assert_energy, assert_grad

pytestmark = pytest.mark.gpu


def _check(batch, insts, energy, grad):
    for i, inst in enumerate(insts):
        e0, g0 = oracle.energy_grad(inst)
        assert_energy(energy[i], e0, inst["ham"], inst["name"])
        a, b = batch.offsets[i], batch.offsets[i + 1]
        assert_grad(grad[a:b], g0, inst["ham"], inst["name"])


def test_h2_sweep_batch():
    insts = W.h2_sweep(100)
    for k, inst in enumerate(insts):
        inst["theta"] = np.array([0.05 * k - 2.0])
    b = svqe.Batch(insts)
    e, g = b.run(b.theta_of(insts))
    _check(b, insts, e, g)


def test_h2_sto3g_sweep_batch():
    """The real molecule (STO-3G, Jordan-Wigner) over the paper's 100 bond lengths."""
    from paper_2601_09951_gb300 import h2_sto3g
    insts = h2_sto3g.h2_sto3g_sweep(100)
    for k, inst in enumerate(insts):
        inst["theta"] = np.array([0.05 * k - 2.0])
    b = svqe.Batch(insts)
    e, g = b.run(b.theta_of(insts))
    _check(b, insts, e, g)


def test_hea_batch_small_sample():
    insts = W.hea_batch(48)
    b = svqe.Batch(insts)
    e, g = b.run(b.theta_of(insts))
    _check(b, insts, e, g)


def test_mixed_gate_batch_with_ragged_sizes():
    insts = [W.uccsd_instance(n=n, n_elec=n // 2, n_singles=6, n_doubles=6, n_terms=60,
                              seed=n) for n in (4, 7, 12)]
    insts += [W.hea_instance(n, 2, 40, n, ring=True) for n in (1, 2, 3, 5, 12)]
    insts += W.h2_sweep(5)
    b = svqe.Batch(insts)
    e, g = b.run(b.theta_of(insts))
    _check(b, insts, e, g)


def test_batching_identity_bitwise():
    insts = W.hea_batch(40)
    big = svqe.Batch(insts)
    e_all, g_all = big.run(big.theta_of(insts))
    for i in (0, 7, 23, 39):
        one = svqe.Batch([insts[i]])
        e1, g1 = one.run(one.theta_of([insts[i]]))
        assert e1[0] == e_all[i]
        a, b = big.offsets[i], big.offsets[i + 1]
        assert np.array_equal(g1, g_all[a:b])
    sub = [insts[j] for j in (39, 3, 17)]
    sb = svqe.Batch(sub)
    es, gs = sb.run(sb.theta_of(sub))
    for k, j in enumerate((39, 3, 17)):
        assert es[k] == e_all[j]


def test_device_buffers_and_graph_replay():
    torch = pytest.importorskip("torch")
    insts = W.hea_batch(16)
    b = svqe.Batch(insts)
    th = torch.tensor(b.theta_of(insts), dtype=torch.float64, device="cuda")
    e = torch.empty(len(insts), dtype=torch.float64, device="cuda")
    g = torch.empty(b.n_params, dtype=torch.float64, device="cuda")
    e_h, g_h = b.run(b.theta_of(insts))
    for _ in range(3):
        b.run_dev(th.data_ptr(), e.data_ptr(), g.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(e.cpu().numpy(), e_h)
    assert np.array_equal(g.cpu().numpy(), g_h)


def test_on_device_gradient_descent_h2():
    torch = pytest.importorskip("torch")
    insts = W.h2_sweep(100)[::20]
    b = svqe.Batch(insts)
    lr, T = 0.4, 50
    th = torch.zeros(len(insts), dtype=torch.float64, device="cuda")
    traj = torch.empty(T, len(insts), dtype=torch.float64, device="cuda")
    b.vqe_dev(th.data_ptr(), lr, T, traj.data_ptr())
    torch.cuda.synchronize()
    traj = traj.cpu().numpy()
    # per-step parity: replay the trajectory one step at a time and check E_t, g_t
    th1 = torch.zeros(len(insts), dtype=torch.float64, device="cuda")
    for t in range(T):
        before = th1.cpu().numpy().copy()
        b.vqe_dev(th1.data_ptr(), lr, 1, None)
        torch.cuda.synchronize()
        after = th1.cpu().numpy()
        for i, inst in enumerate(insts):
            e0, g0 = oracle.energy_grad(inst, before[i:i + 1])
            assert_energy(traj[t, i], e0, inst["ham"], f"{inst['name']} step {t}")
            assert_grad((before[i:i + 1] - after[i:i + 1]) / lr, g0, inst["ham"])
    assert np.array_equal(th.cpu().numpy(), th1.cpu().numpy())


def test_cost_model_counts_by_hand():
    """One H2 instance: DoubleExcitation on 16 amplitudes is 1 pair (12 forward + 24 un-apply
    + 8 gradient flops); two real groups (x = 0 with 11 terms, x = 1111 with 4 two-Y strings)
    at 4 flops per amplitude each, plus 4 per amplitude for the energy: 44 + 128 + 64."""
    b = svqe.Batch(W.h2_sweep(1))
    flops, _ = b.cost()
    assert flops == 44 + 2 * 16 * 4 + 16 * 4


def test_on_device_adam_h2_sweep_paper_settings():
    """The paper's procedure (Sec. 3.4): Adam with alpha = 0.01 from theta = 0, 200 iterations,
    over 100 bond lengths in one launch; per-step energies against the oracle's Adam on
    sampled bonds, and the same trajectory when run one step per call (moments persist)."""
    torch = pytest.importorskip("torch")
    insts = W.h2_sweep(100)
    b = svqe.Batch(insts)
    T = 200
    th = torch.zeros(100, dtype=torch.float64, device="cuda")
    traj = torch.empty(T, 100, dtype=torch.float64, device="cuda")
    b.adam_dev(th.data_ptr(), 0.01, T, traj.data_ptr(), reset=True)
    torch.cuda.synchronize()
    traj = traj.cpu().numpy()
    for i in (0, 37, 74, 99):
        es, _, th_end = oracle.adam_trajectory(insts[i], 0.01, T)
        for t in range(T):
            assert_energy(traj[t, i], es[t], insts[i]["ham"], f"bond {i} step {t}")
        assert abs(th.cpu().numpy()[i] - th_end[0]) <= 1e-9
    th1 = torch.zeros(100, dtype=torch.float64, device="cuda")
    b.adam_dev(th1.data_ptr(), 0.01, 1, None, reset=True)
    for _ in range(T - 1):
        b.adam_dev(th1.data_ptr(), 0.01, 1, None, reset=False)
    torch.cuda.synchronize()
    assert np.array_equal(th1.cpu().numpy(), th.cpu().numpy())


def test_product_layer_from_any_reference_and_partial_layers():
    """A first RY layer on the reference basis state is written directly as a product state.
    Cover references other than |0...0>, first layers that leave qubits out, an RX first layer
    (not a product layer) and one-qubit layers, against the oracle."""
    rng = np.random.default_rng(71)
    insts = []
    for n in (1, 2, 3, 5, 8, 10, 11, 12):
        for variant in range(3):
            cb = W.CircuitBuilder(n)
            qs = list(range(n)) if variant == 0 else [int(q) for q in rng.permutation(n)[: max(1, n - 2)]]
            first = W.RX if variant == 2 else W.RY
            for q in qs:
                cb.add(first, (q,), param="new")
            for q in range(n):
                cb.add(W.RZ, (q,), param="new")
            for q in range(n - 1):
                cb.add(W.CNOT, (q, q + 1))
            for q in range(n):
                cb.add(W.RY, (q,), param="new")
            circ = cb.build()
            insts.append({"circuit": circ, "ham": W.random_pauli_sum(rng, n, 30, 0.6, 3, 1.0),
                          "ref": int(rng.integers(0, 1 << n)),
                          "theta": rng.uniform(-np.pi, np.pi, circ["n_params"]),
                          "name": f"product_n{n}_v{variant}"})
    b = svqe.Batch(insts)
    e, g = b.run(b.theta_of(insts))
    _check(b, insts, e, g)
