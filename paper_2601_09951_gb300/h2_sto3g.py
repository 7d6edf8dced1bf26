"""The paper's molecule as a qubit Hamiltonian: H2 in the STO-3G minimal basis, mapped to four
qubits by Jordan-Wigner (Sec. 2.1, 3.2).

This is an input builder.  It computes the molecular integrals over contracted s-type
Gaussians, takes the restricted Hartree-Fock orbitals (in a minimal basis a homonuclear
diatomic's orbitals are fixed by symmetry: sigma_g and sigma_u), builds the second-quantised
Hamiltonian over spin orbitals, and decomposes it into Pauli strings.  It holds none of the VQE
method's arithmetic (state simulation, energy, gradient), which lives in the CUDA library and,
independently, in the oracle.

Conventions match the rest of the package:
- qubit j is spin orbital j: even j spin up, odd j spin down, spatial orbital j // 2 (sigma_g,
  then sigma_u);
- qubit 0 is the most significant bit of a basis index, and bit value 1 means occupied, so the
  Hartree-Fock state is |1100>;
- a_j = Z_0 ... Z_{j-1} |0><1|_j;
- a Pauli string is a pair of masks (x, z) over basis-index bits, P = i^{popc(x & z)} X^x Z^z.

The integral formulas are the closed forms for s-type Gaussians exp(-a |r - A|^2): overlap,
kinetic energy, nuclear attraction and electron repulsion, the last two through the Boys
function F0.  Energies are in Hartree, lengths in bohr unless named in Angstrom.
"""
import itertools
import math

import numpy as np

from .workloads import DOUBLE_EXC, CircuitBuilder

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903

# STO-3G: the least-squares fit of a Slater 1s function of exponent 1 by three Gaussians
# (Hehre, Stewart and Pople, 1969), as Gaussian exponents and contraction coefficients.  For
# Slater exponent zeta the Gaussian exponents scale by zeta^2; hydrogen in molecules uses
# zeta = 1.24.
STO3G_EXPONENTS_ZETA1 = (2.227660584, 0.405771156, 0.109818)
STO3G_COEFFICIENTS = (0.154328967, 0.535328142, 0.444634542)
ZETA_H_MOLECULE = 1.24


def boys_f0(t):
    """F0(t) = integral_0^1 exp(-t u^2) du = sqrt(pi / t) erf(sqrt t) / 2."""
    if t < 1e-10:
        return 1.0 - t / 3.0
    return 0.5 * math.sqrt(math.pi / t) * math.erf(math.sqrt(t))


def contracted_1s(zeta=ZETA_H_MOLECULE):
    """[(exponent, coefficient x primitive normalisation)] of an STO-3G 1s function."""
    return [(a * zeta * zeta, d * (2.0 * a * zeta * zeta / math.pi) ** 0.75)
            for a, d in zip(STO3G_EXPONENTS_ZETA1, STO3G_COEFFICIENTS)]


def _overlap(a, A, b, B):
    p = a + b
    return (math.pi / p) ** 1.5 * math.exp(-a * b / p * (A - B) ** 2)


def _kinetic(a, A, b, B):
    p = a + b
    mu = a * b / p
    r2 = (A - B) ** 2
    return mu * (3.0 - 2.0 * mu * r2) * (math.pi / p) ** 1.5 * math.exp(-mu * r2)


def _nuclear(a, A, b, B, C, charge):
    p = a + b
    P = (a * A + b * B) / p
    return (-2.0 * math.pi / p * charge * math.exp(-a * b / p * (A - B) ** 2)
            * boys_f0(p * (P - C) ** 2))


def _repulsion(a, A, b, B, c, C, d, D):
    p, q = a + b, c + d
    P, Q = (a * A + b * B) / p, (c * C + d * D) / q
    pref = 2.0 * math.pi ** 2.5 / (p * q * math.sqrt(p + q))
    return (pref * math.exp(-a * b / p * (A - B) ** 2 - c * d / q * (C - D) ** 2)
            * boys_f0(p * q / (p + q) * (P - Q) ** 2))


def ao_integrals(r_bohr, zeta=ZETA_H_MOLECULE):
    """Integrals over the two atomic 1s functions of H2 (nuclei on a line, r_bohr apart):
    overlap S, core Hamiltonian T + V (both nuclei, charge 1) and (ab|cd) (chemists' order)."""
    centres = (0.0, float(r_bohr))
    basis = [[(e, c, X) for e, c in contracted_1s(zeta)] for X in centres]
    S = np.zeros((2, 2))
    Hc = np.zeros((2, 2))
    for i, j in itertools.product(range(2), repeat=2):
        for (a, ca, A), (b, cb, B) in itertools.product(basis[i], basis[j]):
            w = ca * cb
            S[i, j] += w * _overlap(a, A, b, B)
            Hc[i, j] += w * (_kinetic(a, A, b, B)
                             + sum(_nuclear(a, A, b, B, C, 1.0) for C in centres))
    eri = np.zeros((2, 2, 2, 2))
    for i, j, k, l in itertools.product(range(2), repeat=4):
        v = 0.0
        for (a, ca, A), (b, cb, B), (c, cc, C), (d, cd, D) in itertools.product(
                basis[i], basis[j], basis[k], basis[l]):
            v += ca * cb * cc * cd * _repulsion(a, A, b, B, c, C, d, D)
        eri[i, j, k, l] = v
    return S, Hc, eri


def hydrogen_atom_energy(zeta=1.0):
    """Energy of one electron in an STO-3G 1s function on a proton: <phi|T + V|phi>."""
    e = 0.0
    for (a, ca), (b, cb) in itertools.product(contracted_1s(zeta), repeat=2):
        e += ca * cb * (_kinetic(a, 0.0, b, 0.0) + _nuclear(a, 0.0, b, 0.0, 0.0, 1.0))
    return e


def mo_integrals(r_bohr, zeta=ZETA_H_MOLECULE):
    """Core Hamiltonian and (pq|rs) over the restricted Hartree-Fock orbitals sigma_g =
    (phi_A + phi_B) / sqrt(2 (1 + S)) and sigma_u = (phi_A - phi_B) / sqrt(2 (1 - S)); with one
    function per atom and inversion symmetry these are the self-consistent orbitals."""
    S, Hc, eri = ao_integrals(r_bohr, zeta)
    s = S[0, 1]
    C = np.array([[1.0 / math.sqrt(2.0 * (1.0 + s)), 1.0 / math.sqrt(2.0 * (1.0 - s))],
                  [1.0 / math.sqrt(2.0 * (1.0 + s)), -1.0 / math.sqrt(2.0 * (1.0 - s))]])
    h = C.T @ Hc @ C
    g = np.einsum("ap,bq,cr,ds,abcd->pqrs", C, C, C, C, eri)
    return h, g


def _annihilators(n):
    lower = np.array([[0.0, 1.0], [0.0, 0.0]])  # |0><1|
    z = np.diag([1.0, -1.0])
    eye = np.eye(2)
    out = []
    for j in range(n):
        m = np.ones((1, 1))
        for q in range(n):
            m = np.kron(m, z if q < j else lower if q == j else eye)
        out.append(m)
    return out


def fermion_hamiltonian_matrix(r_bohr, zeta=ZETA_H_MOLECULE):
    """The 16 x 16 qubit matrix of H = sum h_ij a+_i a_j + 1/2 sum <ij|kl> a+_i a+_j a_l a_k
    + 1/R over the four spin orbitals, with <ij|kl> = (ik|jl) for matching spins."""
    h, g = mo_integrals(r_bohr, zeta)
    a = _annihilators(4)
    H = np.eye(16) / float(r_bohr)
    for i, j in itertools.product(range(4), repeat=2):
        if i % 2 == j % 2:
            H += h[i // 2, j // 2] * (a[i].T @ a[j])
    for i, j, k, l in itertools.product(range(4), repeat=4):
        if i % 2 == k % 2 and j % 2 == l % 2:
            v = g[i // 2, k // 2, j // 2, l // 2]
            if v != 0.0:
                H += 0.5 * v * (a[i].T @ a[j].T @ a[l] @ a[k])
    return H


def pauli_decomposition(H, n, tol=1e-12):
    """(x, z, c) with H = sum c P(x, z): c = Tr(P H) / 2^n, P[k ^ x, k] =
    i^{popc(x & z)} (-1)^{popc(z & k)}; terms with |c| <= tol are dropped."""
    dim = 1 << n
    k = np.arange(dim)
    terms = []
    for x in range(dim):
        for z in range(dim):
            phase = 1j ** (bin(x & z).count("1") % 4)
            sign = np.array([-1.0 if bin(z & int(kk)).count("1") & 1 else 1.0 for kk in k])
            # Tr(P H) = sum_k P[k ^ x, k] H[k, k ^ x]
            c = phase * np.sum(sign * H[k, k ^ x]) / dim
            if abs(c) > tol:
                if abs(c.imag) > 1e-12:
                    raise ValueError("H is not Hermitian: a Pauli coefficient is complex")
                terms.append((x, z, float(c.real)))
    return terms


def h2_hamiltonian(bond_length_angstrom):
    """The qubit Hamiltonian of H2 at the given bond length: {"n", "x", "z", "coeff"}."""
    r = float(bond_length_angstrom) * BOHR_PER_ANGSTROM
    terms = pauli_decomposition(fermion_hamiltonian_matrix(r), 4)
    return {"n": 4,
            "x": np.array([t[0] for t in terms], dtype=np.uint64),
            "z": np.array([t[1] for t in terms], dtype=np.uint64),
            "coeff": np.array([t[2] for t in terms], dtype=np.float64)}


def h2_sto3g_sweep(n_bonds=100):
    """The paper's sweep with the real molecule: bond k of n_bonds at d = 0.1 + 2.9 k /
    (n_bonds - 1) Angstrom (Sec. 2.2), |HF> = |1100> and one DoubleExcitation(theta) on wires
    (0, 1, 2, 3) (Sec. 3.3), theta starting at 0 (Sec. 3.4)."""
    out = []
    for k in range(n_bonds):
        d = 0.1 + 2.9 * k / max(n_bonds - 1, 1)
        cb = CircuitBuilder(4)
        cb.add(DOUBLE_EXC, (0, 1, 2, 3), param="new")
        out.append({"name": f"h2_sto3g_bond{k}", "bond_length": d, "circuit": cb.build(),
                    "ham": h2_hamiltonian(d), "ref": 0b1100, "theta": np.zeros(1)})
    return out
