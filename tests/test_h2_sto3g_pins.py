"""Pins of the real H2 Hamiltonian (STO-3G, Jordan-Wigner; Sec. 2.1, 3.2) and of the oracle's
VQE energies on it, against values the paper prints, a textbook's worked example, and closed
forms of the integrals.  CPU only.

- Sec. 6.1: at equilibrium the single-parameter VQE energy is about -1.137 Ha and the exact
  STO-3G value is -1.1372 Ha.  Sec. 5.1: the equilibrium bond length is near 0.74 Angstrom and
  the curve flattens into separated atoms beyond 2.5 Angstrom.
- tests/golden/h2_sto3g_r1p4.txt: integrals and energies of the minimal-basis H2 example at
  R = 1.4 bohr (Szabo and Ostlund), to four decimals.
- Closed forms: a normalised Gaussian's overlap, kinetic and nuclear-attraction integrals, the
  point-charge limits of the attraction and repulsion integrals, and F0 by quadrature.
"""
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad

import oracle
from paper_2601_09951_gb300 import h2_sto3g as M
from paper_2601_09951_gb300 import workloads as W
from tests.dense_pins import ham_dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "h2_sto3g_r1p4.txt")


def _golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


# ----------------------------------------------------------------------------- integrals
@pytest.mark.parametrize("t", [0.0, 1e-12, 1e-6, 0.3, 1.0, 7.5, 40.0])
def test_boys_f0_is_the_integral(t):
    want = quad(lambda u: math.exp(-t * u * u), 0.0, 1.0, epsabs=1e-14, epsrel=1e-13)[0]
    assert abs(M.boys_f0(t) - want) <= 1e-12


@pytest.mark.parametrize("alpha", [0.1, 0.62, 3.4, 25.0])
def test_normalised_gaussian_closed_forms(alpha):
    """For g = (2a/pi)^(3/4) exp(-a r^2): <g|g> = 1, <g|-lap/2|g> = 3a/2 and the attraction
    of a unit charge at its centre is -2 sqrt(2a/pi)."""
    n2 = (2.0 * alpha / math.pi) ** 1.5
    assert abs(n2 * M._overlap(alpha, 0.0, alpha, 0.0) - 1.0) <= 1e-14
    assert abs(n2 * M._kinetic(alpha, 0.0, alpha, 0.0) - 1.5 * alpha) <= 1e-13 * alpha
    want = -2.0 * math.sqrt(2.0 * alpha / math.pi)
    assert abs(n2 * M._nuclear(alpha, 0.0, alpha, 0.0, 0.0, 1.0) - want) <= 1e-13 * abs(want)


def test_point_charge_limits():
    """Tight normalised Gaussians act as point charges: attraction -1/R, repulsion 1/R."""
    a, R = 1e8, 1.7
    n2 = (2.0 * a / math.pi) ** 1.5
    assert abs(n2 * M._nuclear(a, 0.0, a, 0.0, R, 1.0) + 1.0 / R) <= 1e-9
    assert abs(n2 * n2 * M._repulsion(a, 0.0, a, 0.0, a, R, a, R) - 1.0 / R) <= 1e-9


def test_sto3g_function_is_normalised_and_scales_like_a_slater_function():
    S, _, _ = M.ao_integrals(1.4)
    assert abs(S[0, 0] - 1.0) <= 2e-6 and abs(S[1, 1] - 1.0) <= 2e-6
    # scaling r -> zeta r: kinetic ~ zeta^2, potential ~ zeta, so E(z) = z^2 T1 + z V1
    e1, e2, e3 = (M.hydrogen_atom_energy(z) for z in (1.0, 1.24, 2.0))
    T1 = (e3 / 2.0 - e1) / (2.0 - 1.0)  # from E(1) = T1 + V1, E(2) = 4 T1 + 2 V1
    V1 = e1 - T1
    assert abs(e2 - (1.24 ** 2 * T1 + 1.24 * V1)) <= 1e-12
    assert -0.5 < e1 < -0.49  # variational, and close to the exact -1/2


def test_textbook_example_at_1p4_bohr():
    g = _golden()
    S, Hc, eri = M.ao_integrals(1.4)
    got = {"S12": S[0, 1], "Hcore11": Hc[0, 0], "Hcore12": Hc[0, 1],
           "eri1111": eri[0, 0, 0, 0], "eri1122": eri[0, 0, 1, 1],
           "eri1212": eri[0, 1, 0, 1], "eri1211": eri[0, 1, 0, 0]}
    H = M.fermion_hamiltonian_matrix(1.4)
    got["E_HF"] = H[0b1100, 0b1100]
    got["E_exact"] = np.linalg.eigvalsh(H)[0]
    for k, v in g.items():
        assert abs(got[k] - v) <= 1e-4, (k, got[k], v)


# ------------------------------------------------------------------------- the Hamiltonian
def test_decomposition_is_exact_and_has_the_h2_structure():
    for d in (0.3, 0.74, 2.0):
        ham = M.h2_hamiltonian(d)
        Hm = M.fermion_hamiltonian_matrix(d * M.BOHR_PER_ANGSTROM)
        assert np.max(np.abs(ham_dense(4, ham) - Hm)) <= 1e-12
        allowed = {W.pauli_masks(4, f) for f in W.H2_STRINGS}
        got = {(int(x), int(z)): c for x, z, c in zip(ham["x"], ham["z"], ham["coeff"])}
        assert set(got) == allowed
        z = {q: W.pauli_masks(4, {q: "Z"}) for q in range(4)}
        # spin symmetry: the two spin orbitals of a spatial orbital are alike
        assert abs(got[z[0]] - got[z[1]]) <= 1e-12 and abs(got[z[2]] - got[z[3]]) <= 1e-12
        # the double-excitation family: XXYY = YYXX = -XYYX = -YXXY
        c = [got[W.pauli_masks(4, dict(zip(range(4), s)))] for s in ("XXYY", "YYXX",
                                                                    "XYYX", "YXXY")]
        assert abs(c[0] - c[1]) <= 1e-12 and abs(c[2] - c[3]) <= 1e-12
        assert abs(c[0] + c[2]) <= 1e-12 and abs(c[0]) > 1e-3


def test_hamiltonian_conserves_particle_number_and_spin():
    Hm = M.fermion_hamiltonian_matrix(1.4)
    nk = np.array([bin(k).count("1") for k in range(16)])
    # S_z: up orbitals are qubits 0 and 2 (bits 3 and 1), down are qubits 1 and 3
    sz = np.array([((k >> 3) & 1) + ((k >> 1) & 1) - ((k >> 2) & 1) - (k & 1)
                   for k in range(16)])
    for lab in (nk, sz):
        mask = lab[:, None] != lab[None, :]
        assert np.max(np.abs(Hm[mask])) == 0.0


# ------------------------------------------------------------------ the paper's energies
def _vqe_minimum(inst):
    """The oracle's energy at the optimum of the one-parameter ansatz: E(t) = a + b cos t +
    c sin t (Sec. 3.3), from three oracle energies; returns (E at the optimum from the
    oracle, a - sqrt(b^2 + c^2))."""
    E = [float(oracle.energy(inst, np.array([t]))) for t in (0.0, math.pi / 2, math.pi)]
    a = 0.5 * (E[0] + E[2])
    b = 0.5 * (E[0] - E[2])
    c = E[1] - a
    t_opt = math.atan2(-c, -b)
    return float(oracle.energy(inst, np.array([t_opt]))), a - math.hypot(b, c)


def test_equilibrium_energy_matches_the_paper():
    """Sec. 6.1: about -1.137 Ha from VQE, -1.1372 Ha exact in STO-3G, near 0.74 Angstrom."""
    ham = M.h2_hamiltonian(0.74)
    exact = np.linalg.eigvalsh(ham_dense(4, ham))[0]
    assert abs(exact - (-1.1372)) <= 1e-4
    cb = W.CircuitBuilder(4)
    cb.add(W.DOUBLE_EXC, (0, 1, 2, 3), param="new")
    inst = {"circuit": cb.build(), "ham": ham, "ref": 0b1100, "theta": np.zeros(1)}
    e_opt, e_closed = _vqe_minimum(inst)
    assert abs(e_opt - e_closed) <= 1e-12
    assert abs(e_opt - (-1.137)) <= 5e-4
    # the one-parameter ansatz spans the exact ground state of minimal-basis H2
    assert abs(e_opt - exact) <= 1e-10
    # the Hartree-Fock state (theta = 0) lies above it
    assert float(oracle.energy(inst, np.zeros(1))) > exact + 0.01


def test_potential_energy_surface_shape():
    """Sec. 5.1: minimum near 0.74 Angstrom, repulsive at short range, flat beyond 2.5
    Angstrom (separated atoms: twice the atom's energy in the same basis)."""
    sweep = M.h2_sto3g_sweep(100)
    E = np.array([_vqe_minimum(inst)[1] for inst in sweep])
    d = np.array([inst["bond_length"] for inst in sweep])
    k = int(np.argmin(E))
    assert abs(d[k] - 0.74) <= 0.03
    assert E[0] > 0.0 and np.all(np.diff(E[:k + 1]) < 0)
    tail = E[d > 2.5]
    assert np.ptp(tail) < 0.01
    assert abs(E[-1] - 2.0 * M.hydrogen_atom_energy(M.ZETA_H_MOLECULE)) < 2e-3
    # every instance starts at theta = 0 on |1100>, with the 15 strings
    assert all(inst["ref"] == 0b1100 and inst["theta"][0] == 0.0 for inst in sweep)
