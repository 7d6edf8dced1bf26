"""Parity at the workloads' full sizes, in the launch configuration the benchmark times.

Where the oracle can compute an output one by one it is compared element by element: sampled
instances of the 4096-instance batch (computed during the test), and, for the single-state
workloads, values the oracle wrote beforehand to tests/golden/ (make_fullsize_golden.py: one
oracle energy takes minutes to hours at these sizes).  Beyond that, properties that hold at
any size are checked: unit norm, |E| <= ||c||_1, and the adjoint gradient against central
differences of the energy."""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2601_09951_gb300 import svqe
from paper_2601_09951_gb300 import workloads as W
from tests.parity import assert_energy, assert_grad, l1

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)
import make_fullsize_golden as MG  # noqa: E402


def _golden(fname, inst):
    """The oracle's stored values for `inst`, refused if the instance arrays differ from the
    ones the values were computed on."""
    g = MG.read_golden(os.path.join(GOLDEN, fname))
    assert g["sha"] == MG.fingerprint(inst), f"{fname} was computed on another instance"
    return g


pytestmark = pytest.mark.gpu


def test_batch_of_4096_sampled_against_oracle():
    insts = W.hea_batch(4096)
    b = svqe.Batch(insts)
    e, g = b.run(b.theta_of(insts))
    for i, inst in enumerate(insts):
        assert np.isfinite(e[i]) and abs(e[i]) <= l1(inst["ham"]) * (1 + 1e-12)
    sample = []
    for n in range(4, 13):  # per qubit count: the first, a middle and the costliest instance
        idx = [i for i, it in enumerate(insts) if it["circuit"]["n"] == n]
        costliest = max(idx, key=lambda i: len(insts[i]["circuit"]["types"]) *
                        len(insts[i]["ham"]["coeff"]))
        sample += sorted({idx[0], idx[len(idx) // 2], costliest})
    for i in sample:
        inst = insts[i]
        e0, g0 = oracle.energy_grad(inst)
        assert_energy(e[i], e0, inst["ham"], inst["name"])
        assert_grad(g[b.offsets[i]:b.offsets[i + 1]], g0, inst["ham"], inst["name"])


def test_h2_sweep_100_bonds_50_steps_on_device():
    torch = pytest.importorskip("torch")
    insts = W.h2_sweep(100)
    b = svqe.Batch(insts)
    lr, T = 0.4, 50
    th = torch.zeros(100, dtype=torch.float64, device="cuda")
    traj = torch.empty(T, 100, dtype=torch.float64, device="cuda")
    b.vqe_dev(th.data_ptr(), lr, T, traj.data_ptr())
    torch.cuda.synchronize()
    traj = traj.cpu().numpy()
    th_final = th.cpu().numpy()
    # per-step parity at the GPU's own theta_t, replayed one step at a time
    th1 = torch.zeros(100, dtype=torch.float64, device="cuda")
    for t in range(T):
        before = th1.cpu().numpy().copy()
        b.vqe_dev(th1.data_ptr(), lr, 1, None)
        torch.cuda.synchronize()
        after = th1.cpu().numpy()
        for i in (0, 33, 66, 99):
            e0, g0 = oracle.energy_grad(insts[i], before[i:i + 1])
            assert_energy(traj[t, i], e0, insts[i]["ham"], f"bond {i} step {t}")
            assert_grad((before[i:i + 1] - after[i:i + 1]) / lr, g0, insts[i]["ham"])
    assert np.array_equal(th1.cpu().numpy(), th_final)
    # the stored energy of every bond: E(theta_final) (Algorithm 1's last line)
    e, _ = b.run(th_final)
    for i in range(100):
        assert_energy(e[i], oracle.energy(insts[i], th_final[i:i + 1]), insts[i]["ham"])


def _single(inst):
    n = inst["circuit"]["n"]
    ctx = svqe.Context(n)
    ctx.init_reference(inst["ref"])
    H = svqe.Ham(ctx, inst["ham"])
    e, g = ctx.adjoint_grad(inst["circuit"], inst["theta"], H)
    return ctx, H, e, g


def test_uccsd_20_qubits_full_gradient():
    """All 400 gradient entries of the 20-qubit UCCSD-shaped circuit against the oracle's
    parameter-shift gradient (four-term rule for the Givens gates), element by element."""
    inst = W.uccsd_instance()
    gold = _golden("uccsd20_oracle.txt", inst)
    ctx, H, e, g = _single(inst)
    assert sorted(gold["grad"]) == list(range(400))
    assert_energy(e, gold["energy"], inst["ham"], "uccsd20")
    assert_grad(g, np.array([gold["grad"][p] for p in range(400)]), inst["ham"], "uccsd20")
    H.close()
    ctx.close()


def test_hea_22_qubits_sampled_gradient():
    inst = W.hea_single(22)
    ctx, H, e, g = _single(inst)
    which = [0, 21, 22, 250, 439]
    e0, g0 = oracle.energy_grad_subset(inst, which)
    assert_energy(e, e0, inst["ham"], "hea22")
    assert_grad(g[which], np.array([g0[p] for p in which]), inst["ham"], "hea22")
    H.close()
    ctx.close()


@pytest.mark.parametrize("n", [24, 26, 28, 30])
def test_hea_full_size_against_stored_oracle_values(n):
    """The 10-layer hardware-efficient circuit with 100 random strings at n qubits: the
    adjoint path's energy and sampled gradient entries against the oracle's stored values."""
    inst = W.hea_single(n)
    gold = _golden(f"hea_single_n{n}_oracle.txt", inst)
    ctx, H, e, g = _single(inst)
    assert_energy(e, gold["energy"], inst["ham"], f"hea{n}")
    ps = sorted(gold["grad"])
    assert_grad(g[ps], np.array([gold["grad"][p] for p in ps]), inst["ham"], f"hea{n}")
    assert abs(e) <= l1(inst["ham"])
    H.close()
    ctx.close()


def test_31_qubits_adjoint_in_three_buffers():
    """31 qubits, 10 layers, 100 strings: the whole adjoint evaluation runs with at most three
    state-sized buffers (the out-of-place diagonal + permutation segments use the third).  Its
    energy matches the oracle's stored value; psi keeps unit norm after the sweep; two gradient
    entries match central differences of sv_expval_paulisum on re-applied circuits."""
    inst = W.hea_single(31)
    gold = _golden("hea_single_n31_oracle.txt", inst)
    assert svqe.ctx_device_bytes(31) <= 3 * svqe.state_bytes(31)
    ctx, H, e, g = _single(inst)
    c = l1(inst["ham"])
    assert_energy(e, gold["energy"], inst["ham"], "hea31")
    ident = svqe.Ham(ctx, {"x": np.array([0], np.uint64), "z": np.array([0], np.uint64),
                           "coeff": np.array([1.0])})
    assert abs(ctx.expval(ident) - 1.0) < 1e-11
    th = np.asarray(inst["theta"], dtype=np.float64)

    def energy(t):
        ctx.init_reference(0)
        ctx.apply_circuit(inst["circuit"], t)
        return ctx.expval(H)

    assert abs(energy(th) - e) <= 1e-12 * c
    h = 1e-4
    for p in (7, 555):
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (energy(tp) - energy(tm)) / (2 * h)
        assert abs(fd - g[p]) <= 1e-6 * c, (p, fd, g[p])
    ident.close()
    H.close()
    ctx.close()
