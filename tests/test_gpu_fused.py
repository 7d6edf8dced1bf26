"""GPU parity of the fused shared-memory passes (registers of >= 14 qubits): gates staged in
tiles of 2^11 amplitudes with the low bits contiguous and the other bits strided, diagonal RZ
runs applied from half tables with factors for RZ gates on bits outside the tile, and the
adjoint sweep's per-thread gradient slots."""
import numpy as np
import pytest

import oracle
from paper_2601_09951_gb300 import svqe
from paper_2601_09951_gb300 import workloads as W
from tests.parity import PSI_TOL, assert_energy, assert_grad

pytestmark = pytest.mark.gpu


def _rand_state(n, rng):
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


def test_single_gates_on_high_middle_and_low_wires():
    n = 15
    rng = np.random.default_rng(1)
    ctx = svqe.Context(n)
    cases = []
    for q in (0, 1, 6, 10, 11, 13, 14):
        for g in (W.X, W.H, W.RX, W.RY, W.RZ):
            cases.append((g, [q]))
    for a, b in ((0, 14), (14, 0), (3, 9), (12, 13), (1, 2)):
        for g in (W.CNOT, W.CZ, W.SINGLE_EXC):
            cases.append((g, [a, b]))
    for w in ((0, 1, 2, 3), (14, 0, 7, 9), (11, 12, 13, 14), (5, 2, 13, 0)):
        cases.append((W.DOUBLE_EXC, list(w)))
    for gtype, wires in cases:
        psi = _rand_state(n, rng)
        t = rng.uniform(-7, 7)
        cb = W.CircuitBuilder(n)
        param = gtype in (W.RX, W.RY, W.RZ, W.SINGLE_EXC, W.DOUBLE_EXC)
        cb.add(gtype, wires, param="new" if param else None)
        circ = cb.build()
        ctx.set_state(psi)
        ctx.apply_circuit(circ, np.array([t]) if param else np.zeros(0))
        got = ctx.get_state()
        want = oracle.apply_gate(psi, n, gtype, wires, t)
        assert np.max(np.abs(got - want)) <= PSI_TOL, (W.GATE_NAMES[gtype], wires)


def test_rz_runs_across_tile_and_outer_bits():
    n = 16
    rng = np.random.default_rng(2)
    cb = W.CircuitBuilder(n)
    for q in range(n):
        cb.add(W.H, (q,))
    for q in rng.permutation(n):
        cb.add(W.RZ, (int(q),), param="new")
    for q in range(0, n, 3):
        cb.add(W.RY, (q,), param="new")
    for q in (15, 0, 7, 8, 3):
        cb.add(W.RZ, (q,), param="new")
    circ = cb.build()
    theta = rng.uniform(-np.pi, np.pi, circ["n_params"])
    inst = {"circuit": circ, "ham": W.random_pauli_sum(rng, n, 40, 0.5, 5, 1.0), "ref": 0,
            "theta": theta}
    ctx = svqe.Context(n)
    ctx.init_reference(0)
    ctx.apply_circuit(circ, theta)
    want = oracle.state(circ, theta, 0)
    assert np.max(np.abs(ctx.get_state() - want)) <= PSI_TOL
    H = svqe.Ham(ctx, inst["ham"])
    e, g = ctx.adjoint_grad(circ, theta, H)
    e0, g0 = oracle.energy_grad(inst)
    assert_energy(e, e0, inst["ham"])
    assert_grad(g, g0, inst["ham"])


@pytest.mark.parametrize("make", [
    lambda: W.hea_instance(16, 2, 60, 31, ring=True),
    lambda: W.hea_instance(14, 3, 80, 32),
    lambda: W.uccsd_instance(n=16, n_elec=8, n_singles=16, n_doubles=24, n_terms=300, seed=33),
])
def test_adjoint_through_fused_passes(make):
    inst = make()
    n = inst["circuit"]["n"]
    ctx = svqe.Context(n)
    ctx.init_reference(inst["ref"])
    H = svqe.Ham(ctx, inst["ham"])
    e, g = ctx.adjoint_grad(inst["circuit"], inst["theta"], H)
    e0, g0 = oracle.energy_grad(inst)
    assert_energy(e, e0, inst["ham"], inst["name"])
    assert_grad(g, g0, inst["ham"], inst["name"])


def test_fused_and_per_op_paths_agree_on_the_state():
    """The same 16-qubit circuit applied as one circuit (fused passes) and gate by gate
    (one-gate circuits, which the planner turns into one-item passes)."""
    inst = W.hea_instance(16, 3, 10, 34, ring=True)
    circ = inst["circuit"]
    ctx = svqe.Context(16)
    ctx.init_reference(0)
    ctx.apply_circuit(circ, inst["theta"])
    fused = ctx.get_state()
    ctx.init_reference(0)
    for gi in range(len(circ["types"])):
        one = {"n": 16, "types": circ["types"][gi:gi + 1], "wires": circ["wires"][gi:gi + 1],
               "params": circ["params"][gi:gi + 1], "fixed": circ["fixed"][gi:gi + 1],
               "n_params": circ["n_params"]}
        ctx.apply_circuit(one, inst["theta"])
    np.testing.assert_allclose(ctx.get_state(), fused, atol=PSI_TOL)


@pytest.mark.parametrize("make,budget_layers", [
    (lambda: W.hea_instance(16, 3, 60, 35, ring=True), 3),
    (lambda: W.hea_instance(14, 4, 80, 36), 2),
    (lambda: W.hea_instance(15, 2, 50, 37), 8),
])
def test_checkpointed_layers_match_oracle_and_plain_sweep(make, budget_layers):
    """With a checkpoint budget, commuting RY layers take their gradients at the layer's end and
    the sweep un-applies them to lambda only, reloading psi.  Energy and gradient match the
    oracle and the sweep without checkpoints, and psi returns to the reference state."""
    inst = make()
    n = inst["circuit"]["n"]
    ctx = svqe.Context(n)
    ctx.init_reference(inst["ref"])
    H = svqe.Ham(ctx, inst["ham"])
    e_plain, g_plain = ctx.adjoint_grad(inst["circuit"], inst["theta"], H)
    ctx.set_checkpoint_bytes(budget_layers * svqe.state_bytes(n))
    e, g = ctx.adjoint_grad(inst["circuit"], inst["theta"], H)
    e0, g0 = oracle.energy_grad(inst)
    assert_energy(e, e0, inst["ham"], inst["name"])
    assert_grad(g, g0, inst["ham"], inst["name"])
    assert abs(e - e_plain) <= 1e-13 * max(1.0, abs(e_plain))
    np.testing.assert_allclose(g, g_plain, rtol=0, atol=1e-11 * max(1.0, np.abs(g_plain).max()))
    ref = np.zeros(1 << n, np.complex128)
    ref[inst["ref"]] = 1.0
    assert np.max(np.abs(ctx.get_state() - ref)) <= 1e-12
    # a second call with the same buffers, then the budget withdrawn
    e2, g2 = ctx.adjoint_grad(inst["circuit"], inst["theta"], H)
    assert e2 == e and np.array_equal(g2, g)
    ctx.set_checkpoint_bytes(0)
    e3, g3 = ctx.adjoint_grad(inst["circuit"], inst["theta"], H)
    assert e3 == e_plain and np.array_equal(g3, g_plain)


def _dp_circuit(n, rng):
    """Runs of RZ and CZ gates followed by CNOT and X runs (whole-state diagonal + permutation
    segments), between single-qubit layers; wires span the low, middle and top bits."""
    cb = W.CircuitBuilder(n)
    for q in range(n):
        cb.add(W.H, (q,))
    for _ in range(3):
        for q in rng.permutation(n)[: n // 2]:
            cb.add(W.RY, (int(q),), param="new")
        for q in rng.permutation(n)[:6]:
            cb.add(W.RZ, (int(q),), param="new")
        cb.add(W.CZ, (0, n - 1))
        cb.add(W.CZ, (3, 7))
        cb.add(W.RZ, (n - 1,), param="new")
        for q in range(n - 1):
            cb.add(W.CNOT, (q, q + 1))
        cb.add(W.CNOT, (n - 1, 0))
        cb.add(W.X, (5,))
        cb.add(W.CNOT, (n - 2, 1))
    return cb.build()


@pytest.mark.parametrize("n,budget", [(14, 0), (15, 2), (16, 0)])
def test_diagonal_permutation_segments(n, budget):
    rng = np.random.default_rng(40 + n)
    circ = _dp_circuit(n, rng)
    theta = rng.uniform(-np.pi, np.pi, circ["n_params"])
    inst = {"circuit": circ, "ham": W.random_pauli_sum(rng, n, 60, 0.5, 4, 1.0), "ref": 6,
            "theta": theta, "name": f"dp_n{n}"}
    ctx = svqe.Context(n)
    ctx.set_checkpoint_bytes(budget * svqe.state_bytes(n))
    # forward alone: the state, in the context's psi buffer
    ctx.init_reference(inst["ref"])
    ctx.apply_circuit(circ, theta)
    want = oracle.state(circ, theta, inst["ref"])
    assert np.max(np.abs(ctx.get_state() - want)) <= PSI_TOL
    # energy and gradient
    ctx.init_reference(inst["ref"])
    H = svqe.Ham(ctx, inst["ham"])
    e, g = ctx.adjoint_grad(circ, theta, H)
    e0, g0 = oracle.energy_grad(inst)
    assert_energy(e, e0, inst["ham"], inst["name"])
    assert_grad(g, g0, inst["ham"], inst["name"])
    ref = np.zeros(1 << n, np.complex128)
    ref[inst["ref"]] = 1.0
    assert np.max(np.abs(ctx.get_state() - ref)) <= 1e-12


def test_tile_size_autotuner(tmp_path, monkeypatch):
    """With autotuning on, the first evaluation of a circuit structure times tiles of 2^9..2^11
    amplitudes and keeps the fastest; the choice is cached for every context of the process
    (and appended to SVQE_TUNE_CACHE), and the result matches the oracle and the default
    tile size."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("SVQE_TUNE_CACHE", str(cache))
    inst = W.uccsd_instance(n=15, n_elec=8, n_singles=12, n_doubles=20, n_terms=200, seed=44)
    n = inst["circuit"]["n"]
    plain = svqe.Context(n)
    plain.init_reference(inst["ref"])
    Hp = svqe.Ham(plain, inst["ham"])
    e_plain, g_plain = plain.adjoint_grad(inst["circuit"], inst["theta"], Hp)
    assert plain.tile_bits() == 11
    ctx = svqe.Context(n)
    ctx.set_autotune(True)
    ctx.init_reference(inst["ref"])
    H = svqe.Ham(ctx, inst["ham"])
    e, g = ctx.adjoint_grad(inst["circuit"], inst["theta"], H)
    bits = ctx.tile_bits()
    assert bits in (9, 10, 11)
    e0, g0 = oracle.energy_grad(inst)
    assert_energy(e, e0, inst["ham"], inst["name"])
    assert_grad(g, g0, inst["ham"], inst["name"])
    assert abs(e - e_plain) <= 1e-12 * max(1.0, abs(e_plain))
    np.testing.assert_allclose(g, g_plain, rtol=0, atol=1e-10 * max(1.0, np.abs(g_plain).max()))
    other = svqe.Context(n)
    other.set_autotune(True)
    other.init_reference(inst["ref"])
    H2 = svqe.Ham(other, inst["ham"])
    e2, g2 = other.adjoint_grad(inst["circuit"], inst["theta"], H2)
    assert other.tile_bits() == bits and e2 == e and np.array_equal(g2, g)
    lines = cache.read_text().split("\n")
    assert any(line.startswith(f"{n} ") and line.endswith(f" {bits}") for line in lines)
