"""Seeded synthetic instance generators (inputs only; no arithmetic of the method).

Both the CUDA path and the CPU oracle read what these functions return and nothing else; this
module computes no state, gate, energy or gradient.  Every instance is a plain dict:

    {"name": str,
     "circuit": {"n": n_qubits, "types": int32[G], "wires": int32[G, 4] (-1 padded),
                 "params": int32[G] (-1 = fixed angle), "fixed": float64[G], "n_params": P},
     "ham": {"x": uint64[T], "z": uint64[T], "coeff": float64[T]},
     "ref": basis index of the reference state,
     "theta": float64[P]}

Conventions of the format: qubit q is bit (n-1-q) of a basis index (qubit 0 is the most
significant bit, so |1100> = 12); a Pauli string is a pair of masks over basis-index bits,
x = bits where the factor is X or Y, z = bits where it is Z or Y.

Shapes follow the paper's workloads (Sec. 2.2: 100 bond lengths on [0.1, 3.0] A; Sec. 3.3: HF
reference and one DoubleExcitation on 4 qubits; Sec. 3.2: a Jordan-Wigner Pauli sum; Sec. 5.2:
a qubit-count scaling study).  The coefficients here are synthetic; the real H2/STO-3G
Hamiltonian over the same bond lengths comes from ``h2_sto3g.py``.
"""
import itertools
import math

import numpy as np

# Gate codes of the instance format.
X, H, RX, RY, RZ, CNOT, SINGLE_EXC, DOUBLE_EXC, CZ = range(9)
GATE_NAMES = {X: "X", H: "H", RX: "RX", RY: "RY", RZ: "RZ", CNOT: "CNOT",
              SINGLE_EXC: "SingleExcitation", DOUBLE_EXC: "DoubleExcitation", CZ: "CZ"}
N_WIRES = {X: 1, H: 1, RX: 1, RY: 1, RZ: 1, CNOT: 2, SINGLE_EXC: 2, DOUBLE_EXC: 4, CZ: 2}


def _rng(seed, *stream):
    return np.random.Generator(np.random.PCG64([int(seed), *[int(s) for s in stream]]))


def pauli_masks(n, factors):
    """Masks (x, z) of the Pauli string {qubit: 'X'|'Y'|'Z'} on n qubits."""
    x = z = 0
    for q, p in factors.items():
        if not 0 <= q < n:
            raise ValueError("qubit out of range")
        b = 1 << (n - 1 - q)
        if p in ("X", "Y"):
            x |= b
        if p in ("Z", "Y"):
            z |= b
    return x, z


class CircuitBuilder:
    """Accumulates gate records in the instance format."""

    def __init__(self, n):
        self.n = n
        self.types, self.wires, self.params, self.fixed = [], [], [], []
        self.n_params = 0

    def add(self, gtype, wires, param=None, angle=0.0):
        w = list(wires) + [-1] * (4 - len(wires))
        self.types.append(gtype)
        self.wires.append(w)
        if param == "new":
            param = self.n_params
            self.n_params += 1
        self.params.append(-1 if param is None else int(param))
        self.fixed.append(float(angle))
        return self.params[-1]

    def build(self):
        return {"n": self.n,
                "types": np.array(self.types, dtype=np.int32),
                "wires": np.array(self.wires, dtype=np.int32).reshape(-1, 4),
                "params": np.array(self.params, dtype=np.int32),
                "fixed": np.array(self.fixed, dtype=np.float64),
                "n_params": self.n_params}


def _ham(terms):
    x = np.array([t[0] for t in terms], dtype=np.uint64)
    z = np.array([t[1] for t in terms], dtype=np.uint64)
    c = np.array([t[2] for t in terms], dtype=np.float64)
    return {"x": x, "z": z, "coeff": c}


# ----------------------------------------------------------------------------------------
# Workload 1: H2-shaped sweep, 4 qubits, 100 bond lengths.
# ----------------------------------------------------------------------------------------
H2_STRINGS = ([{}] + [{q: "Z"} for q in range(4)]
              + [{a: "Z", b: "Z"} for a in range(4) for b in range(a + 1, 4)]
              + [dict(zip(range(4), s)) for s in ("XXYY", "YYXX", "XYYX", "YXXY")])


def h2_sweep(n_bonds=100, seed=1001):
    """The H2-shaped sweep: |HF> = |1100>, one DoubleExcitation(theta) on wires (0,1,2,3),
    15 Jordan-Wigner-structured terms (I; Z0..Z3; six ZiZj; XXYY, YYXX, XYYX, YXXY).  Per term
    two draws u0, u1 ~ U[-1, 1]; bond k of n_bonds has s = k/(n_bonds-1) and coefficients
    (1-s)*u0 + s*u1, labelled with d = 0.1 + 2.9*s Angstrom.  theta starts at 0."""
    rng = _rng(seed)
    u0 = rng.uniform(-1.0, 1.0, size=len(H2_STRINGS))
    u1 = rng.uniform(-1.0, 1.0, size=len(H2_STRINGS))
    masks = [pauli_masks(4, f) for f in H2_STRINGS]
    out = []
    for k in range(n_bonds):
        s = k / max(n_bonds - 1, 1)
        coeff = (1.0 - s) * u0 + s * u1
        cb = CircuitBuilder(4)
        cb.add(DOUBLE_EXC, (0, 1, 2, 3), param="new")
        out.append({"name": f"h2_bond{k}", "bond_length": 0.1 + 2.9 * s,
                    "circuit": cb.build(),
                    "ham": _ham([(x, z, c) for (x, z), c in zip(masks, coeff)]),
                    "ref": 0b1100, "theta": np.zeros(1)})
    return out


# ----------------------------------------------------------------------------------------
# Workload 2: batched small hardware-efficient circuits.
# ----------------------------------------------------------------------------------------
def random_pauli_sum(rng, n, n_terms, p_zonly, max_weight, sigma, allow_identity=True):
    """n_terms strings: with probability p_zonly an I/Z-only string, else one with at least
    one X or Y; weight uniform in [1 (0 for Z-only if allow_identity), max_weight] on
    distinct random wires; coefficients N(0, sigma)."""
    terms = []
    for _ in range(n_terms):
        zonly = rng.random() < p_zonly
        lo = 0 if (zonly and allow_identity) else 1
        w = int(rng.integers(lo, min(max_weight, n) + 1))
        wires = rng.choice(n, size=w, replace=False)
        if zonly:
            f = {int(q): "Z" for q in wires}
        else:
            while True:
                ps = rng.choice(["X", "Y", "Z"], size=w)
                if any(p != "Z" for p in ps):
                    break
            f = {int(q): str(p) for q, p in zip(wires, ps)}
        x, z = pauli_masks(n, f)
        terms.append((x, z, float(rng.normal(0.0, sigma))))
    return _ham(terms)


def hea_circuit(n, layers, ring=False):
    """Hardware-efficient ansatz: per layer RY on every qubit, RZ on every qubit, then a CNOT
    ladder q -> q+1 (plus n-1 -> 0 when ring=True).  Parameters are numbered in gate order."""
    cb = CircuitBuilder(n)
    for _ in range(layers):
        for q in range(n):
            cb.add(RY, (q,), param="new")
        for q in range(n):
            cb.add(RZ, (q,), param="new")
        for q in range(n - 1):
            cb.add(CNOT, (q, q + 1))
        if ring and n > 2:
            cb.add(CNOT, (n - 1, 0))
    return cb.build()


def hea_instance(n, layers, n_terms, seed, stream=0, p_zonly=0.7, max_weight=4, sigma=0.5,
                 ring=False, name=None):
    rng = _rng(seed, stream)
    circ = hea_circuit(n, layers, ring=ring)
    theta = rng.uniform(-np.pi, np.pi, size=circ["n_params"])
    ham = random_pauli_sum(rng, n, n_terms, p_zonly, max_weight, sigma)
    return {"name": name or f"hea_n{n}_L{layers}_T{n_terms}", "circuit": circ, "ham": ham,
            "ref": 0, "theta": theta}


def hea_batch_spec(i, seed=1002):
    """(n, L, T) of instance i of the batched workload: n ~ U{4..12}, L ~ U{2..8},
    T ~ U{50..500}."""
    rng = _rng(seed, i, 0)
    return int(rng.integers(4, 13)), int(rng.integers(2, 9)), int(rng.integers(50, 501))


def hea_batch(n_inst=4096, seed=1002, indices=None):
    """The batched workload: n_inst independent instances, each from its own seeded stream so
    any subset can be regenerated alone.  Z-heavy Hamiltonians: 70% I/Z-only strings, weight
    <= 4, coefficients N(0, 0.5); parameters U[-pi, pi]; reference |0...0>."""
    idx = range(n_inst) if indices is None else indices
    out = []
    for i in idx:
        n, L, T = hea_batch_spec(i, seed)
        inst = hea_instance(n, L, T, seed, stream=i + 1, name=f"batch{i}_n{n}_L{L}_T{T}")
        inst["index"] = int(i)
        out.append(inst)
    return out


# ----------------------------------------------------------------------------------------
# Workload 3: 20-qubit UCCSD-shaped circuit.
# ----------------------------------------------------------------------------------------
def uccsd_instance(n=20, n_elec=10, n_singles=80, n_doubles=320, n_terms=2000, seed=1003):
    """HF reference with qubits 0..n_elec-1 occupied; n_doubles DoubleExcitation gates (i, j ->
    a, b) then n_singles SingleExcitation gates (i -> a), spin conserving (even qubit = alpha,
    odd = beta), drawn with replacement; parameters N(0, 0.1).  Wires are ordered (occupied...,
    virtual...), so the HF pattern on a gate's wires is |10> / |1100>.

    Hamiltonian of n_terms weight <= 4 strings: I, every Z_i, every Z_iZ_j, then 8-string
    families on seeded p<q<r<s (all X/Y strings with an even number of Y), then X_pX_q+Y_pY_q
    pairs, topped up with single X_pX_q strings to exactly n_terms (fewer on registers too
    small to hold that many distinct strings).  Coefficients +-1/(1+rank), rank a seeded
    permutation."""
    rng = _rng(seed)
    occ = list(range(n_elec))
    vir = list(range(n_elec, n))
    cb = CircuitBuilder(n)
    for _ in range(n_doubles):
        while True:
            i, j = sorted(rng.choice(occ, size=2, replace=False))
            a, b = sorted(rng.choice(vir, size=2, replace=False))
            if sorted([i % 2, j % 2]) == sorted([a % 2, b % 2]):
                break
        cb.add(DOUBLE_EXC, (int(i), int(j), int(a), int(b)), param="new")
    for _ in range(n_singles):
        while True:
            i = int(rng.choice(occ))
            a = int(rng.choice(vir))
            if i % 2 == a % 2:
                break
        cb.add(SINGLE_EXC, (i, a), param="new")
    circ = cb.build()
    theta = rng.normal(0.0, 0.1, size=circ["n_params"])

    strings = [{}]
    strings += [{q: "Z"} for q in range(n)]
    strings += [{p: "Z", q: "Z"} for p in range(n) for q in range(p + 1, n)]
    fam8 = [s for s in ("".join(t) for t in itertools.product("XY", repeat=4))
            if s.count("Y") % 2 == 0]
    remaining = n_terms - len(strings)
    n_quads = min(max(remaining, 0) // 8, 180, math.comb(n, 4))
    quads = set()
    while len(quads) < n_quads:
        quads.add(tuple(sorted(int(v) for v in rng.choice(n, size=4, replace=False))))
    for qd in sorted(quads):
        for s in sorted(fam8):
            strings.append(dict(zip(qd, s)))
    remaining = n_terms - len(strings)
    n_pairs = min(max(remaining, 0) // 2, n * (n - 1) // 2)
    pairs = set()
    while len(pairs) < n_pairs:
        pairs.add(tuple(sorted(int(v) for v in rng.choice(n, size=2, replace=False))))
    for p, q in sorted(pairs):
        strings.append({p: "X", q: "X"})
        strings.append({p: "Y", q: "Y"})
    free = [pq for pq in itertools.combinations(range(n), 2) if pq not in pairs]
    rng.shuffle(free)
    while len(strings) < n_terms and free:
        p, q = free.pop()
        strings.append({p: "X", q: "X"})
    strings = strings[:n_terms]
    rank = rng.permutation(len(strings))
    sign = rng.choice([-1.0, 1.0], size=len(strings))
    terms = [pauli_masks(n, f) + (float(sign[k] / (1.0 + rank[k])),)
             for k, f in enumerate(strings)]
    ref = sum(1 << (n - 1 - q) for q in occ)
    return {"name": f"uccsd_n{n}", "circuit": circ, "ham": _ham(terms), "ref": ref,
            "theta": theta}


# ----------------------------------------------------------------------------------------
# Workload 4: single-state scaling sweep.
# ----------------------------------------------------------------------------------------
def hea_single(n, layers=10, n_terms=100, seed=1004):
    """|0..0>, `layers` layers of RY(all), RZ(all), CNOT ring; parameters U[-pi, pi]; n_terms
    random strings of weight U{1..6} on distinct wires, factors U{X, Y, Z}, coefficients
    N(0, 1)."""
    rng = _rng(seed, n)
    circ = hea_circuit(n, layers, ring=True)
    theta = rng.uniform(-np.pi, np.pi, size=circ["n_params"])
    terms = []
    for _ in range(n_terms):
        w = int(rng.integers(1, min(6, n) + 1))
        wires = rng.choice(n, size=w, replace=False)
        ps = rng.choice(["X", "Y", "Z"], size=w)
        x, z = pauli_masks(n, {int(q): str(p) for q, p in zip(wires, ps)})
        terms.append((x, z, float(rng.normal(0.0, 1.0))))
    return {"name": f"hea_single_n{n}", "circuit": circ, "ham": _ham(terms), "ref": 0,
            "theta": theta}


# ----------------------------------------------------------------------------------------
# Workload 6: the scaling study's transverse-field Ising Hamiltonian (Sec. 5.2, Table 3).
# ----------------------------------------------------------------------------------------
def tfim_instance(n, layers=2, J=1.0, h=1.0, seed=1006):
    """H = -J sum_i Z_i Z_{i+1} - h sum_i X_i on an open chain of n qubits (the paper names
    its scaling-study Hamiltonian both a sum of Pauli-Z operators and a transverse-field Ising
    model; the Ising form contains the Z sum).  Ansatz: `layers` layers of RY(all), RZ(all),
    CNOT ladder from |0..0>; parameters U[-pi, pi] from the seeded stream of n."""
    rng = _rng(seed, n)
    circ = hea_circuit(n, layers)
    theta = rng.uniform(-np.pi, np.pi, size=circ["n_params"])
    terms = []
    for i in range(n - 1):
        x, z = pauli_masks(n, {i: "Z", i + 1: "Z"})
        terms.append((x, z, -float(J)))
    for i in range(n):
        x, z = pauli_masks(n, {i: "X"})
        terms.append((x, z, -float(h)))
    return {"name": f"tfim_n{n}_L{layers}", "circuit": circ, "ham": _ham(terms), "ref": 0,
            "theta": theta}


# ----------------------------------------------------------------------------------------
# Workload 5: serving stream.
# ----------------------------------------------------------------------------------------
def serve_stream(n_requests, rate_per_s, seed=1005, max_qubits=24, steps=20):
    """Poisson arrivals at `rate_per_s`; n = round(4 * 6^u), u ~ U[0, 1] (log-uniform on
    [4, 24]); n == 4 gives an H2-shaped request at a random bond, otherwise a hardware-
    efficient request shaped like the batched workload.  Each request asks for `steps`
    gradient-descent steps with step 0.4 / ||c||_1."""
    rng = _rng(seed)
    t = 0.0
    out = []
    h2 = None
    for r in range(n_requests):
        t += float(rng.exponential(1.0 / rate_per_s))
        n = int(round(4 * 6 ** rng.random()))
        n = max(4, min(n, max_qubits))
        if n == 4:
            if h2 is None:
                h2 = h2_sweep(100, seed=seed + 1)
            inst = dict(h2[int(rng.integers(0, 100))])
        else:
            L, T = int(rng.integers(2, 9)), int(rng.integers(50, 501))
            inst = hea_instance(n, L, T, seed, stream=r + 1)
        inst = dict(inst)
        inst["name"] = f"req{r}_n{n}"
        inst["arrival_s"] = t
        inst["steps"] = steps
        inst["lr"] = 0.4 / float(np.abs(inst["ham"]["coeff"]).sum())
        out.append(inst)
    return out
