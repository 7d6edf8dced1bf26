"""Pins of the CPU oracle against what the paper and the mathematics fix (CPU only).

Each check reaches the answer by a route that shares nothing with the oracle's code:
dense Kronecker/expm matrices, Jordan-Wigner fermion operators for Eq. 5, the hand-derived
closed form of the one-parameter H2 ansatz, exact diagonalisation (variational bound, Eq. 2),
central finite differences, and textbook special cases.
"""
import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from paper_2601_09951_gb300 import workloads as W
from tests import dense_pins as D


def _rand_state(n, rng):
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


# ------------------------------------------------------------------ single gates vs dense
@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_one_qubit_gates_match_expm(n):
    rng = np.random.default_rng(10 + n)
    for gtype in (W.X, W.H, W.RX, W.RY, W.RZ):
        for q in range(n):
            t = rng.uniform(-7, 7)
            psi = _rand_state(n, rng)
            got = oracle.apply_gate(psi, n, gtype, [q], t)
            want = D.gate_dense(n, gtype, [q], t) @ psi
            np.testing.assert_allclose(got, want, atol=1e-14, rtol=0)


@pytest.mark.parametrize("n", [2, 3, 5])
def test_two_qubit_gates_match_dense(n):
    rng = np.random.default_rng(20 + n)
    for gtype in (W.CNOT, W.CZ, W.SINGLE_EXC):
        for a in range(n):
            for b in range(n):
                if a == b:
                    continue
                t = rng.uniform(-7, 7)
                psi = _rand_state(n, rng)
                got = oracle.apply_gate(psi, n, gtype, [a, b], t)
                want = D.gate_dense(n, gtype, [a, b], t) @ psi
                np.testing.assert_allclose(got, want, atol=1e-14, rtol=0)


@pytest.mark.parametrize("n", [4, 6])
def test_double_excitation_matches_dense(n):
    rng = np.random.default_rng(30 + n)
    for _ in range(12):
        wires = [int(w) for w in rng.choice(n, size=4, replace=False)]
        t = rng.uniform(-7, 7)
        psi = _rand_state(n, rng)
        got = oracle.apply_gate(psi, n, W.DOUBLE_EXC, wires, t)
        want = D.gate_dense(n, W.DOUBLE_EXC, wires, t) @ psi
        np.testing.assert_allclose(got, want, atol=1e-14, rtol=0)


def test_double_excitation_is_eq5_with_jordan_wigner():
    """Eq. 5 with its imaginary unit dropped (as printed, exp(-i t/2 (A - A^dag)) with A - A^dag
    anti-Hermitian is not unitary): U(t) = exp(-t/2 (A - A^dag)), A = a0^dag a1^dag a2 a3 under
    Jordan-Wigner a_j = Z_0..Z_{j-1}|0><1|_j.  That is the oracle's DoubleExcitation on
    wires (0, 1, 2, 3)."""
    n = 4
    a = [D.annihilator(n, j) for j in range(n)]
    A = a[0].conj().T @ a[1].conj().T @ a[2] @ a[3]
    rng = np.random.default_rng(5)
    for t in [0.3, -1.1, np.pi, 2.5]:
        U = expm(-0.5 * t * (A - A.conj().T))
        np.testing.assert_allclose(U @ U.conj().T, np.eye(16), atol=1e-13)
        for _ in range(3):
            psi = _rand_state(n, rng)
            got = oracle.apply_gate(psi, n, W.DOUBLE_EXC, [0, 1, 2, 3], t)
            np.testing.assert_allclose(got, U @ psi, atol=1e-14, rtol=0)


# ------------------------------------------------------------------ Pauli-sum energy vs dense
@pytest.mark.parametrize("n", [1, 3, 6, 8])
def test_expval_matches_dense_hamiltonian(n):
    rng = np.random.default_rng(40 + n)
    ham = W.random_pauli_sum(rng, n, 40, 0.5, min(4, n), 0.7)
    Hd = D.ham_dense(n, ham)
    psi = _rand_state(n, rng)
    re, im = oracle.expval(psi, n, ham)
    want = np.vdot(psi, Hd @ psi)
    assert abs(re - want.real) <= 1e-13 * max(1.0, np.abs(ham["coeff"]).sum())
    assert abs(im) <= 1e-13 * max(1.0, np.abs(ham["coeff"]).sum())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_energy_matches_dense_circuit(seed):
    """Whole circuits: oracle E(theta) vs psi^dag H psi with U built from dense gates."""
    for inst in [W.hea_instance(5, 3, 30, seed, ring=True),
                 W.hea_instance(7, 2, 60, seed + 100),
                 W.uccsd_instance(n=8, n_elec=4, n_singles=6, n_doubles=6, n_terms=80,
                                  seed=seed)]:
        circ = inst["circuit"]
        n = circ["n"]
        U = D.circuit_dense(circ, inst["theta"])
        ref = np.zeros(1 << n, dtype=complex)
        ref[inst["ref"]] = 1
        psi = U @ ref
        np.testing.assert_allclose(oracle.state(circ, inst["theta"], inst["ref"]), psi,
                                   atol=1e-13, rtol=0)
        Hd = D.ham_dense(n, inst["ham"])
        want = np.vdot(psi, Hd @ psi).real
        got = oracle.energy(inst)
        assert abs(got - want) <= 1e-12 * np.abs(inst["ham"]["coeff"]).sum()


# ------------------------------------------------------------------ closed form of workload 1
def _h2_closed_form_abc(coeff):
    """Hand derivation (Sec. 3.3): psi(t) = cos(t/2)|1100> - sin(t/2)|0011>, so
    E(t) = a + b cos t + c sin t with a = (H_AA + H_BB)/2, b = (H_AA - H_BB)/2, c = -H_AB.
    Z_q is -1 on an occupied qubit.  A = |1100> (qubits 0, 1 occupied), B = |0011>.
    <A|P|B> for the four flip strings, from Y|0> = i|1> and Y|1> = -i|0>:
    XXYY: (-i)(-i) = -1; YYXX: (i)(i) = -1; XYYX: (i)(-i) = 1; YXXY: (i)(-i) = 1."""
    cI, cz, czz, cf = coeff[0], coeff[1:5], coeff[5:11], coeff[11:15]
    zA = [-1, -1, 1, 1]
    zB = [1, 1, -1, -1]
    pairs = [(a, b) for a in range(4) for b in range(a + 1, 4)]
    HAA = cI + sum(c * z for c, z in zip(cz, zA)) + sum(
        c * zA[a] * zA[b] for c, (a, b) in zip(czz, pairs))
    HBB = cI + sum(c * z for c, z in zip(cz, zB)) + sum(
        c * zB[a] * zB[b] for c, (a, b) in zip(czz, pairs))
    HAB = -cf[0] - cf[1] + cf[2] + cf[3]
    return (HAA + HBB) / 2, (HAA - HBB) / 2, -HAB


def test_h2_structure_is_the_jordan_wigner_string_set():
    names = []
    for x, z in zip(W.h2_sweep(1)[0]["ham"]["x"], W.h2_sweep(1)[0]["ham"]["z"]):
        s = ""
        for q in range(4):
            b = 1 << (3 - q)
            s += "Y" if (x & b and z & b) else "X" if x & b else "Z" if z & b else "I"
        names.append(s)
    assert names == ["IIII", "ZIII", "IZII", "IIZI", "IIIZ", "ZZII", "ZIZI", "ZIIZ", "IZZI",
                     "IZIZ", "IIZZ", "XXYY", "YYXX", "XYYX", "YXXY"]


def test_h2_energy_and_gradient_closed_form():
    sweep = W.h2_sweep(100)
    rng = np.random.default_rng(7)
    for inst in sweep[::7]:
        a, b, c = _h2_closed_form_abc(inst["ham"]["coeff"])
        for t in np.concatenate([[0.0, np.pi / 2, np.pi], rng.uniform(-4, 4, 3)]):
            e, g = oracle.energy_grad(inst, np.array([t]))
            assert abs(e - (a + b * np.cos(t) + c * np.sin(t))) <= 1e-14 * 16
            assert abs(g[0] - (-b * np.sin(t) + c * np.cos(t))) <= 1e-14 * 16


def test_h2_golden_values():
    """Fixture tests/golden/h2_closed_form.txt: hand-evaluated a, b, c for fixed coefficients."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "h2_closed_form.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    coeff = np.array([float(v) for v in rows[0]])
    a, b, c = (float(v) for v in rows[1])
    inst = W.h2_sweep(1)[0]
    inst = dict(inst, ham=dict(inst["ham"], coeff=coeff))
    for t in [0.0, 0.7, -2.0]:
        e, g = oracle.energy_grad(inst, np.array([t]))
        assert abs(e - (a + b * np.cos(t) + c * np.sin(t))) < 1e-14
        assert abs(g[0] - (-b * np.sin(t) + c * np.cos(t))) < 1e-14


# ------------------------------------------------------------------ variational bound (Eq. 2)
def test_variational_bound():
    rng = np.random.default_rng(11)
    for inst in W.h2_sweep(100)[::10]:
        lam = np.linalg.eigvalsh(D.ham_dense(4, inst["ham"]))[0]
        a, b, c = _h2_closed_form_abc(inst["ham"]["coeff"])
        assert a - np.hypot(b, c) >= lam - 1e-12
        for t in rng.uniform(-np.pi, np.pi, 5):
            assert oracle.energy(inst, np.array([t])) >= lam - 1e-12
    for seed in range(3):
        inst = W.hea_instance(6, 3, 50, seed)
        lam = np.linalg.eigvalsh(D.ham_dense(6, inst["ham"]))[0]
        for _ in range(4):
            th = rng.uniform(-np.pi, np.pi, inst["circuit"]["n_params"])
            assert oracle.energy(inst, th) >= lam - 1e-12


# ------------------------------------------------------------------ gradient (Algorithm 1)
def _fd_grad(inst, theta, h=1e-5):
    g = np.zeros_like(theta)
    for p in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        g[p] = (oracle.energy(inst, tp) - oracle.energy(inst, tm)) / (2 * h)
    return g


@pytest.mark.parametrize("which", ["hea", "hea_ring", "uccsd"])
def test_parameter_shift_matches_finite_differences(which):
    if which == "uccsd":
        inst = W.uccsd_instance(n=8, n_elec=4, n_singles=8, n_doubles=8, n_terms=120, seed=3)
    else:
        inst = W.hea_instance(6, 2, 60, 4, ring=(which == "hea_ring"))
    e, g = oracle.energy_grad(inst)
    gfd = _fd_grad(inst, inst["theta"].copy())
    scale = np.abs(inst["ham"]["coeff"]).sum()
    np.testing.assert_allclose(g, gfd, atol=2e-8 * scale, rtol=0)


def test_two_term_rule_is_not_enough_for_excitations():
    """The excitation generators have eigenvalues {-1/2, 0, 1/2}; the two-term +-pi/2 rule
    misses the frequency-1/2 part once the state leaves the rotated plane."""
    inst = W.uccsd_instance(n=6, n_elec=2, n_singles=3, n_doubles=2, n_terms=60, seed=9)
    th = inst["theta"] + 0.8
    _, g = oracle.energy_grad(inst, th)
    two_term = []
    for p in range(len(th)):
        tp, tm = th.copy(), th.copy()
        tp[p] += np.pi / 2
        tm[p] -= np.pi / 2
        two_term.append(0.5 * (oracle.energy(inst, tp) - oracle.energy(inst, tm)))
    gfd = _fd_grad(inst, th)
    np.testing.assert_allclose(g, gfd, atol=1e-7)
    assert np.max(np.abs(np.array(two_term) - gfd)) > 1e-4


def test_shared_parameter_sums_occurrences():
    cb = W.CircuitBuilder(3)
    p = cb.add(W.RY, (0,), param="new")
    cb.add(W.RX, (1,), param=p)
    cb.add(W.CNOT, (0, 2))
    cb.add(W.RZ, (2,), param=p)
    cb.add(W.SINGLE_EXC, (1, 2), param=p)
    rng = np.random.default_rng(2)
    inst = {"circuit": cb.build(), "ham": W.random_pauli_sum(rng, 3, 20, 0.3, 3, 1.0),
            "ref": 0b001, "theta": np.array([0.37])}
    _, g = oracle.energy_grad(inst)
    np.testing.assert_allclose(g, _fd_grad(inst, inst["theta"].copy()), atol=1e-8)


# ------------------------------------------------------------------ invariants
def test_norm_and_inverse_round_trip():
    rng = np.random.default_rng(12)
    for inst in [W.hea_instance(8, 4, 10, 1, ring=True),
                 W.uccsd_instance(n=10, n_elec=4, n_singles=10, n_doubles=10, n_terms=20,
                                  seed=2)]:
        circ = inst["circuit"]
        n = circ["n"]
        psi0 = _rand_state(n, rng)
        psi = oracle.apply_circuit(psi0, circ, inst["theta"])
        assert abs(np.linalg.norm(psi) - 1) < 1e-13 * len(circ["types"])
        back = psi
        for g in reversed(range(len(circ["types"]))):
            gt = int(circ["types"][g])
            k = W.N_WIRES[gt]
            p = circ["params"][g]
            t = inst["theta"][p] if p >= 0 else circ["fixed"][g]
            back = oracle.apply_gate(back, n, gt, list(circ["wires"][g][:k]), -t)
        np.testing.assert_allclose(back, psi0, atol=1e-13)


def test_particle_number_conserved_by_givens_circuits():
    inst = W.uccsd_instance(n=10, n_elec=4, n_singles=12, n_doubles=12, n_terms=10, seed=5)
    psi = oracle.state(inst["circuit"], inst["theta"], inst["ref"])
    weights = np.array([bin(i).count("1") for i in range(1 << 10)])
    assert np.all(psi[weights != 4] == 0)
    assert abs(np.linalg.norm(psi) - 1) < 1e-13


def test_special_cases():
    one = oracle.apply_gate(oracle.basis_state(1, 0), 1, W.RY, [0], np.pi)
    np.testing.assert_allclose(one, [0, 1], atol=1e-15)
    de = oracle.apply_gate(oracle.basis_state(4, 0b1100), 4, W.DOUBLE_EXC, [0, 1, 2, 3], np.pi)
    want = np.zeros(16)
    want[0b0011] = -1
    np.testing.assert_allclose(de, want, atol=1e-15)
    plus = oracle.apply_gate(oracle.basis_state(1, 0), 1, W.H, [0])
    assert abs(oracle.expval(plus, 1, {"x": np.array([1], np.uint64),
                                       "z": np.array([0], np.uint64),
                                       "coeff": np.array([1.0])})[0] - 1) < 1e-15
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = 5
        b = int(rng.integers(0, 32))
        z = int(rng.integers(0, 32))
        e, _ = oracle.expval(oracle.basis_state(n, b), n, {"x": np.array([0], np.uint64),
                                                           "z": np.array([z], np.uint64),
                                                           "coeff": np.array([1.0])})
        assert e == (-1.0) ** bin(b & z).count("1")


def test_malformed_gates_rejected():
    psi = oracle.basis_state(3, 0)
    for gtype, wires in [(W.RY, [3]), (W.CNOT, [1, 1]), (W.DOUBLE_EXC, [0, 1, 2, 2]), (99, [0])]:
        with pytest.raises(ValueError):
            oracle.apply_gate(psi, 3, gtype, wires, 0.1)


def test_uccsd_generator_shape():
    inst = W.uccsd_instance()
    assert inst["circuit"]["n"] == 20 and len(inst["circuit"]["types"]) == 400
    assert len(inst["ham"]["coeff"]) == 2000
    assert inst["ref"] == int("1" * 10 + "0" * 10, 2)
    assert np.sum(inst["circuit"]["types"] == W.DOUBLE_EXC) == 320
    pairs = set(zip(inst["ham"]["x"].tolist(), inst["ham"]["z"].tolist()))
    assert len(pairs) == 2000


def test_gradient_subset_equals_full_sweep_entries():
    inst = W.uccsd_instance(n=8, n_elec=4, n_singles=6, n_doubles=6, n_terms=80, seed=12)
    e, g = oracle.energy_grad(inst)
    es, gs = oracle.energy_grad_subset(inst, [0, 5, 11])
    assert es == e
    for p, v in gs.items():
        assert v == g[p]


def test_adam_first_step_and_scale_invariance():
    """Adam's first update is lr * g / (|g| + eps) per parameter (m_hat = g, v_hat = g^2),
    and scaling H (hence g) by a constant leaves the trajectory unchanged up to eps."""
    inst = W.hea_instance(5, 2, 30, 61)
    es, ths, _ = oracle.adam_trajectory(inst, 0.01, 3)
    _, g = oracle.energy_grad(inst)
    step1 = ths[1] - ths[0] if len(ths) > 1 else None
    np.testing.assert_allclose(step1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    big = dict(inst, ham=dict(inst["ham"], coeff=10.0 * inst["ham"]["coeff"]))
    es10, ths10, _ = oracle.adam_trajectory(big, 0.01, 3)
    np.testing.assert_allclose(ths10, ths, atol=1e-7)
    np.testing.assert_allclose(es10, 10 * es, rtol=1e-6, atol=1e-9)


def _stub_gradients(monkeypatch, grads):
    """Make oracle.energy_grad return grads[k] on its k-th call (energy = k), so that the
    optimizer's own arithmetic is all that the trajectory shows."""
    calls = []

    def fake(inst, theta=None):
        k = len(calls)
        calls.append(np.array(theta, dtype=np.float64))
        return float(k), np.array(grads[k], dtype=np.float64)

    monkeypatch.setattr(oracle, "energy_grad", fake)
    return calls


def test_adam_constant_gradient_steps_by_lr_at_every_step(monkeypatch):
    """With a constant gradient g, m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2, so the two
    bias corrections give m_hat = g and v_hat = g^2 at every t (Kingma & Ba; the paper's
    optimizer, Sec. 3.4) and every step is exactly -lr * g / (|g| + eps).  A bias correction
    with a fixed exponent (1 - b^1 at every t) or a dropped one moves every step after the
    first away from this value."""
    g = np.array([0.3, -2.0, 1e-3, 7.5])
    T, lr = 50, 0.01
    inst = {"theta": np.array([0.1, -0.2, 0.3, 0.0])}
    calls = _stub_gradients(monkeypatch, [g] * T)
    es, ths, th_end = oracle.adam_trajectory(inst, lr, T)
    assert len(calls) == T and np.array_equal(es, np.arange(T, dtype=float))
    steps = np.diff(np.vstack([ths, th_end]), axis=0)
    want = -lr * g / (np.abs(g) + 1e-8)
    for t in range(T):
        np.testing.assert_allclose(steps[t], want, rtol=1e-12, atol=0, err_msg=f"step {t + 1}")
    for t in range(T):  # the gradient is evaluated at theta_t, before the update
        assert np.array_equal(calls[t], ths[t])


def test_adam_hand_computed_second_and_third_steps(monkeypatch):
    """Steps 2 and 3 for gradients whose sign or size changes, worked by hand with
    b1 = 0.9, b2 = 0.999 (per parameter, g0 = the first gradient):
      signs +g0, -g0, +g0:
        m1 = 0.1 g0;  m2 = 0.09 g0 - 0.1 g0 = -0.01 g0;  m3 = -0.009 g0 + 0.1 g0 = 0.091 g0
        m_hat2 = -0.01/(1 - 0.81) g0 = -g0/19;  m_hat3 = 0.091/(1 - 0.729) g0 = 91/271 g0
        v_t = (1 - 0.999^t) g0^2, so v_hat = g0^2 and step_t = -lr m_hat_t / (|g0| + eps);
      sizes g0, 2 g0:
        m2 = 0.09 g0 + 0.2 g0 = 0.29 g0, m_hat2 = 29/19 g0
        v2 = 0.999 * 0.001 g0^2 + 0.001 * 4 g0^2 = 0.004999 g0^2,
        v_hat2 = 0.004999 / (1 - 0.998001) g0^2 = 4999/1999 g0^2
        step2 = -lr (29/19) g0 / (sqrt(4999/1999) |g0| + eps)."""
    lr, eps = 0.01, 1e-8
    g0 = np.array([0.5, -1.25, 3.0])
    inst = {"theta": np.zeros(3)}
    _stub_gradients(monkeypatch, [g0, -g0, g0])
    _, ths, th_end = oracle.adam_trajectory(inst, lr, 3)
    steps = np.diff(np.vstack([ths, th_end]), axis=0)
    np.testing.assert_allclose(steps[1], -lr * (-1.0 / 19.0) * g0 / (np.abs(g0) + eps),
                               rtol=1e-12)
    np.testing.assert_allclose(steps[2], -lr * (91.0 / 271.0) * g0 / (np.abs(g0) + eps),
                               rtol=1e-12)
    _stub_gradients(monkeypatch, [g0, 2 * g0])
    _, ths, th_end = oracle.adam_trajectory(inst, lr, 2)
    steps = np.diff(np.vstack([ths, th_end]), axis=0)
    want = -lr * (29.0 / 19.0) * g0 / (np.sqrt(4999.0 / 1999.0) * np.abs(g0) + eps)
    np.testing.assert_allclose(steps[1], want, rtol=1e-12)


def test_gd_trajectory_follows_the_h2_closed_form():
    """Gradient descent on the one-parameter H2 ansatz (the configured bond-length loop:
    step 0.4, 50 steps from theta = 0).  With E = a + b cos t + c sin t (hand-derived above),
    every recorded step is (E(theta_t), E'(theta_t), theta_t) and theta_{t+1} =
    theta_t - 0.4 (-b sin theta_t + c cos theta_t).  The iteration is checked one step at a
    time from the oracle's own theta_t, so that the chaotic bonds (0.4 |E''| > 2) are pinned
    as tightly as the contracting ones; where the map contracts, the whole closed-form
    trajectory is followed as well."""
    lr, T = 0.4, 50
    for inst in W.h2_sweep(100)[::3]:
        a, b, c = _h2_closed_form_abc(inst["ham"]["coeff"])
        es, gs, ths, th_end = oracle.gd_trajectory(inst, lr, T, theta0=np.zeros(1))
        assert es.shape == (T,) and gs.shape == (T, 1) and ths.shape == (T, 1)
        assert ths[0, 0] == 0.0
        nxt = np.concatenate([ths[1:, 0], th_end])
        for t in range(T):
            th = ths[t, 0]
            assert abs(es[t] - (a + b * np.cos(th) + c * np.sin(th))) <= 1e-13
            gc = -b * np.sin(th) + c * np.cos(th)
            assert abs(gs[t, 0] - gc) <= 1e-13
            assert abs(nxt[t] - (th - lr * gc)) <= 1e-13
        R = np.hypot(b, c)
        if abs(1 - lr * R) < 0.9:
            th = 0.0
            for t in range(T):
                th = th - lr * (-b * np.sin(th) + c * np.cos(th))
            assert abs(th - th_end[0]) <= 1e-9


def test_tfim_workload_is_the_ising_chain_and_respects_the_variational_bound():
    """The scaling study's Hamiltonian generator gives -J sum Z_i Z_{i+1} - h sum X_i on an open
    chain (built here from Kronecker products), and the oracle's energy of its ansatz state
    lies above the chain's ground energy (exact diagonalisation)."""
    n, J, h = 5, 1.0, 0.7
    inst = W.tfim_instance(n, J=J, h=h)
    want = sum(-J * D.on_qubits(n, {i: D.PZ, i + 1: D.PZ}) for i in range(n - 1))
    want = want + sum(-h * D.on_qubits(n, {i: D.PX}) for i in range(n))
    got = D.ham_dense(n, inst["ham"])
    np.testing.assert_allclose(got, want, atol=1e-14)
    lam_min = np.linalg.eigvalsh(want)[0]
    e, _ = oracle.energy_grad(inst)
    assert e >= lam_min - 1e-12
