"""GPU parity of the single-state path (sv_init_reference, sv_apply_circuit,
sv_expval_paulisum, sv_adjoint_grad, vqe_step) against the CPU oracle."""
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


def _one_gate(n, gtype, wires, param=True):
    cb = W.CircuitBuilder(n)
    cb.add(gtype, wires, param="new" if param else None)
    return cb.build()


@pytest.mark.parametrize("n", [1, 2, 3, 6, 11])
def test_every_gate_on_every_wire(n):
    rng = np.random.default_rng(100 + n)
    ctx = svqe.Context(n)
    cases = []
    for q in range(n):
        for g in (W.X, W.H, W.RX, W.RY, W.RZ):
            cases.append((g, [q]))
    for a in range(n):
        for b in range(n):
            if a != b:
                for g in (W.CNOT, W.CZ, W.SINGLE_EXC):
                    cases.append((g, [a, b]))
    if n >= 4:
        for _ in range(12):
            cases.append((W.DOUBLE_EXC, [int(w) for w in rng.choice(n, 4, replace=False)]))
    for gtype, wires in cases:
        psi = _rand_state(n, rng)
        t = rng.uniform(-7, 7)
        circ = _one_gate(n, gtype, wires, param=gtype in (W.RX, W.RY, W.RZ, W.SINGLE_EXC,
                                                          W.DOUBLE_EXC))
        th = np.array([t]) if circ["n_params"] else np.zeros(0)
        ctx.set_state(psi)
        ctx.apply_circuit(circ, th)
        got = ctx.get_state()
        want = oracle.apply_gate(psi, n, gtype, wires, t)
        err = np.max(np.abs(got - want))
        assert err <= PSI_TOL, (W.GATE_NAMES[gtype], wires, err)


@pytest.mark.parametrize("inst_fn", [
    lambda: W.hea_instance(10, 4, 80, 1, ring=True),
    lambda: W.uccsd_instance(n=12, n_elec=6, n_singles=20, n_doubles=40, n_terms=300, seed=4),
    lambda: W.h2_sweep(3)[1],
])
def test_circuit_state_and_energy(inst_fn):
    inst = inst_fn()
    n = inst["circuit"]["n"]
    ctx = svqe.Context(n)
    ctx.init_reference(inst["ref"])
    ctx.apply_circuit(inst["circuit"], inst["theta"])
    got = ctx.get_state()
    want = oracle.state(inst["circuit"], inst["theta"], inst["ref"])
    assert np.max(np.abs(got - want)) <= PSI_TOL
    H = svqe.Ham(ctx, inst["ham"])
    assert_energy(ctx.expval(H), oracle.expval(want, n, inst["ham"])[0], inst["ham"])


@pytest.mark.parametrize("n", [1, 2, 5, 9, 14, 20])
def test_expval_random_states_and_groups(n):
    rng = np.random.default_rng(200 + n)
    ham = W.random_pauli_sum(rng, n, 150, 0.3, min(6, n), 1.0)
    # groups with several terms of mixed Y parity (complex tables)
    for s in ("XY", "YX", "XX", "YY", "XZ"):
        f = {q: p for q, p in zip(range(n), s)}
        x, z = W.pauli_masks(n, f)
        ham["x"] = np.append(ham["x"], np.uint64(x))
        ham["z"] = np.append(ham["z"], np.uint64(z))
        ham["coeff"] = np.append(ham["coeff"], rng.normal())
    ctx = svqe.Context(n)
    H = svqe.Ham(ctx, ham)
    for _ in range(3):
        psi = _rand_state(n, rng)
        ctx.set_state(psi)
        assert_energy(ctx.expval(H), oracle.expval(psi, n, ham)[0], ham, f"n={n}")


# One Hamiltonian per group class of the energy kernel: a one-term diagonal group, a
# diagonal table, one-term real / imaginary off-diagonal groups, and real, imaginary and
# complex tables (several strings sharing one X mask).
_CLASS_CASES = {
    "Z": [({0: "Z"}, 0.7)],
    "Z-table": [({0: "Z"}, 0.7), ({1: "Z"}, -0.4), ({0: "Z", 1: "Z"}, 0.25), ({}, 0.1)],
    "XX": [({0: "X", 1: "X"}, 0.9)],
    "Y": [({0: "Y"}, -1.3)],
    "XX+YY": [({0: "X", 1: "X"}, 0.6), ({0: "Y", 1: "Y"}, 0.45)],
    "XY-YX": [({0: "X", 1: "Y"}, 0.8), ({0: "Y", 1: "X"}, -0.35)],
    "X+Y": [({0: "X"}, 0.5), ({0: "Y"}, 0.75)],
}


def _ham_of(n, terms, shift):
    xs, zs, cs = [], [], []
    for f, c in terms:
        x, z = W.pauli_masks(n, {(q + shift) % n: p for q, p in f.items()})
        xs.append(x)
        zs.append(z)
        cs.append(c)
    return {"n": n, "x": np.array(xs, np.uint64), "z": np.array(zs, np.uint64),
            "coeff": np.array(cs, np.float64)}


@pytest.mark.parametrize("case", sorted(_CLASS_CASES))
@pytest.mark.parametrize("n", [2, 3, 8, 9, 16])
def test_expval_each_group_class(case, n):
    """Every class of group, on the top wires, the bottom wires (bit 0) and in between; n = 8
    is one chunk of pairs per group, n = 16 many."""
    rng = np.random.default_rng(300 + n)
    ctx = svqe.Context(n)
    for shift in sorted({0, n // 2, n - 2}):
        ham = _ham_of(n, _CLASS_CASES[case], shift)
        H = svqe.Ham(ctx, ham)
        psi = _rand_state(n, rng)
        ctx.set_state(psi)
        assert_energy(ctx.expval(H), oracle.expval(psi, n, ham)[0], ham,
                      f"{case} n={n} shift={shift}")


@pytest.mark.parametrize("n", [1, 2, 3])
def test_expval_single_qubit_registers(n):
    """n = 1: the diagonal group pairs amplitudes 0 and 1; every group is a single pair."""
    rng = np.random.default_rng(400 + n)
    ctx = svqe.Context(n)
    for case in ("Z", "Y", "X+Y"):
        ham = _ham_of(n, [({q % n: p for q, p in f.items()}, c) for f, c in _CLASS_CASES[case]
                          if all(q < n for q in f)], 0)
        if len(ham["x"]) == 0:
            continue
        H = svqe.Ham(ctx, ham)
        psi = _rand_state(n, rng)
        ctx.set_state(psi)
        assert_energy(ctx.expval(H), oracle.expval(psi, n, ham)[0], ham, f"{case} n={n}")


def _check_adjoint(inst, theta=None):
    theta = inst["theta"] if theta is None else theta
    n = inst["circuit"]["n"]
    ctx = svqe.Context(n)
    ctx.init_reference(inst["ref"])
    H = svqe.Ham(ctx, inst["ham"])
    e, g = ctx.adjoint_grad(inst["circuit"], theta, H)
    e0, g0 = oracle.energy_grad(inst, theta)
    assert_energy(e, e0, inst["ham"], inst.get("name", ""))
    assert_grad(g, g0, inst["ham"], inst.get("name", ""))
    return e, g


@pytest.mark.parametrize("which", ["h2", "hea6", "hea_ring9", "uccsd10", "mixed"])
def test_adjoint_gradient_matches_parameter_shift(which):
    if which == "h2":
        for inst in W.h2_sweep(100)[::33]:
            for t in (0.0, 0.9, -2.4):
                _check_adjoint(inst, np.array([t]))
        return
    if which == "hea6":
        inst = W.hea_instance(6, 3, 60, 7)
    elif which == "hea_ring9":
        inst = W.hea_instance(9, 2, 120, 8, ring=True)
    elif which == "uccsd10":
        inst = W.uccsd_instance(n=10, n_elec=4, n_singles=12, n_doubles=16, n_terms=200, seed=6)
    else:
        cb = W.CircuitBuilder(5)
        p = cb.add(W.RX, (0,), param="new")
        cb.add(W.H, (1,))
        cb.add(W.RY, (1,), param=p)
        cb.add(W.CZ, (1, 3))
        cb.add(W.RZ, (4,), param="new")
        cb.add(W.X, (2,))
        cb.add(W.SINGLE_EXC, (2, 4), param="new")
        cb.add(W.CNOT, (4, 0))
        cb.add(W.DOUBLE_EXC, (3, 1, 0, 2), param=p)
        cb.add(W.RY, (3,), angle=0.77)
        rng = np.random.default_rng(5)
        inst = {"circuit": cb.build(), "ham": W.random_pauli_sum(rng, 5, 60, 0.4, 4, 1.0),
                "ref": 0b10110, "theta": np.array([0.3, -1.2, 2.2])}
    _check_adjoint(inst)


def test_adjoint_restores_nothing_it_should_not():
    """Two calls in a row give bit-identical results (psi is re-initialised from |ref>)."""
    inst = W.hea_instance(8, 3, 90, 11)
    ctx = svqe.Context(8)
    ctx.init_reference(0)
    H = svqe.Ham(ctx, inst["ham"])
    a = ctx.adjoint_grad(inst["circuit"], inst["theta"], H)
    b = ctx.adjoint_grad(inst["circuit"], inst["theta"], H)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_vqe_step_per_step_parity():
    inst = W.h2_sweep(100)[40]
    ctx = svqe.Context(4)
    ctx.init_reference(inst["ref"])
    H = svqe.Ham(ctx, inst["ham"])
    lr, T = 0.4, 50
    theta = np.zeros(1)
    traj = []
    for t in range(T):
        new, es = ctx.vqe_step(inst["circuit"], H, theta, lr, 1)
        e0, g0 = oracle.energy_grad(inst, theta)
        assert_energy(es[0], e0, inst["ham"], f"step {t}")
        assert_grad((theta - new) / lr, g0, inst["ham"], f"step {t}")
        traj.append(es[0])
        theta = new
    # the same 50 steps in one call give the identical trajectory
    th_all, es_all = ctx.vqe_step(inst["circuit"], H, np.zeros(1), lr, T)
    assert np.array_equal(es_all, np.array(traj))
    assert np.array_equal(th_all, theta)


def test_malformed_input_is_einval():
    ctx = svqe.Context(3)
    bad = [
        {"n": 3, "types": [W.RY], "wires": [[3, -1, -1, -1]], "params": [0], "fixed": [0.0],
         "n_params": 1},
        {"n": 3, "types": [W.CNOT], "wires": [[1, 1, -1, -1]], "params": [-1], "fixed": [0.0],
         "n_params": 0},
        {"n": 3, "types": [42], "wires": [[0, -1, -1, -1]], "params": [-1], "fixed": [0.0],
         "n_params": 0},
        {"n": 3, "types": [W.RZ], "wires": [[0, -1, -1, -1]], "params": [5], "fixed": [0.0],
         "n_params": 1},
        {"n": 4, "types": [W.RZ], "wires": [[0, -1, -1, -1]], "params": [0], "fixed": [0.0],
         "n_params": 1},
    ]
    for c in bad:
        with pytest.raises(svqe.SvError) as e:
            ctx.apply_circuit(c, np.zeros(c["n_params"]))
        assert e.value.status == svqe.SV_EINVAL
    with pytest.raises(svqe.SvError) as e:
        svqe.Ham(ctx, {"x": np.array([8], np.uint64), "z": np.array([0], np.uint64),
                       "coeff": np.array([1.0])})
    assert e.value.status == svqe.SV_EINVAL
    with pytest.raises(svqe.SvError):
        ctx.init_reference(8)
    # the context is still usable afterwards
    ctx.init_reference(5)
    assert abs(ctx.get_state()[5] - 1) == 0


@pytest.mark.parametrize("n", [5, 9, 15])
def test_tfim_scaling_workload(n):
    """The scaling study's transverse-field Ising chain under the 2-layer ansatz: energy and
    gradient against the oracle (n = 15 runs the fused and whole-state segment path), and a
    gradient-descent run that lowers the energy."""
    inst = W.tfim_instance(n)
    ctx = svqe.Context(n)
    ctx.init_reference(0)
    H = svqe.Ham(ctx, inst["ham"])
    e, g = ctx.adjoint_grad(inst["circuit"], inst["theta"], H)
    e0, g0 = oracle.energy_grad(inst)
    assert_energy(e, e0, inst["ham"], inst["name"])
    assert_grad(g, g0, inst["ham"], inst["name"])
    _, es = ctx.vqe_step(inst["circuit"], H, inst["theta"], 0.05, 30)
    assert es[-1] < es[0]
