"""Independent dense-matrix constructions used to pin the oracle (tests only).

Nothing here calls the oracle or shares its code path: gate matrices come from matrix
exponentials of their generators (scipy.linalg.expm), multi-qubit operators from Kronecker
products of 2x2 matrices, and the excitation generators from Jordan-Wigner fermion matrices.
Qubit 0 is the leftmost Kronecker factor (the most significant bit of a basis index).
"""
from functools import reduce

import numpy as np
from scipy.linalg import expm

I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
P0 = np.array([[1, 0], [0, 0]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)
LOWER = np.array([[0, 1], [0, 0]], dtype=complex)  # |0><1|: removes an occupation
PAULI = {"I": I2, "X": PX, "Y": PY, "Z": PZ}


def kron_all(ops):
    return reduce(np.kron, ops)


def on_qubits(n, mapping):
    """Kronecker product with mapping {qubit: 2x2} and identity elsewhere."""
    return kron_all([mapping.get(q, I2) for q in range(n)])


def pauli_string_dense(n, masks):
    """Dense matrix of the string with masks over basis-index bits (bit n-1-q <-> qubit q)."""
    x, z = int(masks[0]), int(masks[1])
    ops = []
    for q in range(n):
        b = 1 << (n - 1 - q)
        xb, zb = bool(x & b), bool(z & b)
        ops.append(PY if (xb and zb) else PX if xb else PZ if zb else I2)
    return kron_all(ops)


def ham_dense(n, ham):
    Hd = np.zeros((1 << n, 1 << n), dtype=complex)
    for x, z, c in zip(ham["x"], ham["z"], ham["coeff"]):
        Hd += c * pauli_string_dense(n, (x, z))
    return Hd


def annihilator(n, j):
    """Jordan-Wigner a_j = Z_0 ... Z_{j-1} |0><1|_j."""
    return on_qubits(n, {**{k: PZ for k in range(j)}, j: LOWER})


def givens_generator(n, lo_pattern, hi_pattern, wires):
    """Real antisymmetric K = |hi><lo| - |lo><hi| on the given wires (identity on the rest
    of the register, zero on other patterns of the wires)."""
    dim = 1 << n
    K = np.zeros((dim, dim))
    for i in range(dim):
        bits = [(i >> (n - 1 - w)) & 1 for w in wires]
        if tuple(bits) == tuple(lo_pattern):
            j = i
            for w, lb, hb in zip(wires, lo_pattern, hi_pattern):
                if lb != hb:
                    j ^= 1 << (n - 1 - w)
            K[j, i] += 1.0
            K[i, j] -= 1.0
    return K


def gate_dense(n, gtype, wires, t):
    """Dense unitary of one gate, built from generators and projectors."""
    from paper_2601_09951_gb300 import workloads as W
    if gtype == W.X:
        return on_qubits(n, {wires[0]: PX})
    if gtype == W.H:
        return on_qubits(n, {wires[0]: (PX + PZ) / np.sqrt(2)})
    if gtype in (W.RX, W.RY, W.RZ):
        P = {W.RX: PX, W.RY: PY, W.RZ: PZ}[gtype]
        return on_qubits(n, {wires[0]: expm(-0.5j * t * P)})
    if gtype == W.CNOT:
        c, tq = wires[0], wires[1]
        return on_qubits(n, {c: P0}) + on_qubits(n, {c: P1, tq: PX})
    if gtype == W.CZ:
        a, b = wires[0], wires[1]
        return np.eye(1 << n) - 2 * on_qubits(n, {a: P1, b: P1})
    if gtype == W.SINGLE_EXC:
        K = givens_generator(n, (0, 1), (1, 0), wires[:2])
        return expm(0.5 * t * K)
    if gtype == W.DOUBLE_EXC:
        K = givens_generator(n, (0, 0, 1, 1), (1, 1, 0, 0), wires[:4])
        return expm(0.5 * t * K)
    raise ValueError(gtype)


def circuit_dense(circuit, theta):
    n = circuit["n"]
    U = np.eye(1 << n, dtype=complex)
    for g in range(len(circuit["types"])):
        p = circuit["params"][g]
        t = theta[p] if p >= 0 else circuit["fixed"][g]
        k = {0: 1, 1: 1, 2: 1, 3: 1, 4: 1, 5: 2, 6: 2, 7: 4, 8: 2}[int(circuit["types"][g])]
        U = gate_dense(n, int(circuit["types"][g]), [int(w) for w in circuit["wires"][g][:k]],
                       t) @ U
    return U
