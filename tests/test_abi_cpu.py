"""CPU-only checks of the C ABI: the library loads, exports every declared symbol, and its
host-side logic (sizes, validation, X-mask grouping with Walsh-Hadamard tables) is right.
No compute call needs a GPU here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2601_09951_gb300 import svqe
from paper_2601_09951_gb300 import workloads as W
from tests import dense_pins as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2601_09951_gb300 import build
    build.build()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b((?:sv|vqe)_\w+)\s*\(", src, re.M):
                names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert {"sv_init_reference", "sv_apply_circuit", "sv_expval_paulisum", "sv_adjoint_grad",
            "vqe_step", "sv_batch_run"} <= names
    L = ctypes.CDLL(svqe.lib_path())
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def test_state_sizes_match_table3():
    """Fixture tests/golden/table3_state_bytes.txt: Table 3's state-vector column."""
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden",
                                                 "table3_state_bytes.txt"))
            if l.strip() and not l.startswith("#")]
    unit = {"B": 1, "KB": 1 << 10, "MB": 1 << 20, "GB": 1 << 30}
    for n, val, u in rows:
        assert svqe.state_bytes(int(n)) == int(val) * unit[u]
    # Two state buffers for 31 qubits fit in HBM with room for a third.
    assert svqe.ctx_device_bytes(31) < 3 * svqe.state_bytes(31)
    assert svqe.state_bytes(-1) == 0 and svqe.ctx_device_bytes(32) == 0


def test_status_strings_and_version():
    L = svqe.lib()
    assert L.sv_abi_version() == 1
    assert L.sv_status_str(1) == b"SV_EINVAL"


def test_bad_qubit_count_is_einval_without_touching_the_gpu():
    for n in (0, 32, -3):
        with pytest.raises(svqe.SvError) as e:
            svqe.Context(n)
        assert e.value.status == svqe.SV_EINVAL


def test_context_options_reject_null_handles():
    """sv_set_checkpoint_bytes, sv_set_autotune and sv_tile_bits answer SV_EINVAL for a NULL
    handle (or output) without touching the device."""
    import ctypes
    L = svqe.lib()
    assert L.sv_set_checkpoint_bytes(None, 1 << 30) == svqe.SV_EINVAL
    assert L.sv_set_autotune(None, 1) == svqe.SV_EINVAL
    t = ctypes.c_int32(0)
    assert L.sv_tile_bits(None, ctypes.byref(t)) == svqe.SV_EINVAL
    assert L.sv_tile_bits(None, None) == svqe.SV_EINVAL


def _group_f(n, lowered, g):
    """f_g(k) for every k, from the lowered group record and table."""
    x, zu, cls, toff, table = lowered
    ks = np.arange(1 << n, dtype=np.uint64)
    if cls[g] >= 4:  # one term: coefficient times the parity sign of z & k
        par = np.array([bin(int(k) & int(zu[g])).count("1") & 1 for k in ks])
        return table[toff[g]] * (1 - 2 * par)
    idx = np.zeros(1 << n, dtype=np.int64)
    m, b = int(zu[g]), 0
    while m:
        pos = (m & -m).bit_length() - 1
        idx |= (((ks >> np.uint64(pos)) & np.uint64(1)).astype(np.int64)) << b
        b += 1
        m &= m - 1
    return table[toff[g] + idx]


def _apply_lowered(n, lowered, psi):
    x = lowered[0]
    out = np.zeros_like(psi)
    ks = np.arange(1 << n, dtype=np.uint64)
    for g in range(len(x)):
        out += _group_f(n, lowered, g) * psi[(ks ^ x[g]).astype(np.int64)]
    return out


@pytest.mark.parametrize("n,kmax", [(3, 3), (6, 2), (6, 6), (9, 4)])
def test_grouped_tables_reproduce_dense_h_psi(n, kmax):
    rng = np.random.default_rng(n * 10 + kmax)
    ham = W.random_pauli_sum(rng, n, 120, 0.4, min(4, n), 1.0)
    # several terms sharing one X mask with mixed Y parity (complex tables)
    for s in ("XYZ", "YXZ", "XXZ", "YYI"):
        f = {q: p for q, p in enumerate(s) if p != "I"}
        x, z = W.pauli_masks(n, f)
        ham["x"] = np.append(ham["x"], np.uint64(x))
        ham["z"] = np.append(ham["z"], np.uint64(z))
        ham["coeff"] = np.append(ham["coeff"], rng.normal())
    lowered = svqe.ham_lower(ham, n, kmax)
    widest = max(bin(int(z)).count("1") for z in ham["z"])
    assert np.all([bin(int(z)).count("1") <= max(kmax, widest) for z in lowered[1]])
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    want = D.ham_dense(n, ham) @ psi
    np.testing.assert_allclose(_apply_lowered(n, lowered, psi), want, atol=1e-12)
    # groups share no X mask with a different class than their table needs
    for g, c in enumerate(lowered[2]):
        size = 1 if c >= 4 else 1 << bin(int(lowered[1][g])).count("1")
        t = lowered[4][lowered[3][g]: lowered[3][g] + size]
        if c & 3 == 0:
            assert np.all(t.imag == 0)
        if c & 3 == 1:
            assert np.all(t.real == 0)
    if n >= 6:  # registers this wide leave most X masks with a single term
        assert any(c >= 4 for c in lowered[2]) and any(c < 4 for c in lowered[2])


@pytest.mark.parametrize("n", [1, 4, 7])
def test_lowered_groups_are_hermitian_and_pair_sums_give_the_energy(n):
    """The energy-only kernel visits one member k of each pair (k, k ^ x_g), the one with the
    top bit of x_g clear, and adds 2 Re(conj(psi_k) f_g(k) psi_{k ^ x_g}); the diagonal group
    pairs k with k + N/2.  That needs f_g(k ^ x_g) = conj f_g(k) from the lowered tables.  The
    same summation in NumPy must give psi^H H psi."""
    rng = np.random.default_rng(700 + n)
    ham = W.random_pauli_sum(rng, n, 80, 0.4, min(4, n), 1.0)
    lowered = svqe.ham_lower(ham, n, 4)
    x = lowered[0]
    N = 1 << n
    ks = np.arange(N, dtype=np.int64)
    psi = rng.normal(size=N) + 1j * rng.normal(size=N)
    e = 0.0
    for g in range(len(x)):
        f = _group_f(n, lowered, g)
        xg = int(x[g])
        xp = xg if xg else N >> 1
        np.testing.assert_allclose(f[ks ^ xg], np.conj(f), rtol=1e-14, atol=1e-14)
        h = xp.bit_length() - 1
        lo = (1 << h) - 1
        t = np.arange(N >> 1, dtype=np.int64)
        k = ((t & ~lo) << 1) | (t & lo)
        v, w = psi[k], psi[k ^ xp]
        if xg == 0:
            e += np.sum(f[k].real * np.abs(v) ** 2 + f[k ^ xp].real * np.abs(w) ** 2)
        else:
            e += 2.0 * np.sum((np.conj(v) * f[k] * w).real)
    want = np.vdot(psi, D.ham_dense(n, ham) @ psi).real
    assert abs(e - want) <= 1e-12 * max(1.0, abs(want))


def test_lowering_rejects_bad_masks():
    with pytest.raises(svqe.SvError) as e:
        svqe.ham_lower({"x": np.array([8], np.uint64), "z": np.array([0], np.uint64),
                        "coeff": np.array([1.0])}, 3, 3)
    assert e.value.status == svqe.SV_EINVAL


def _gate_bits(circ, g):
    k = W.N_WIRES[int(circ["types"][g])]
    return {int(circ["n"]) - 1 - int(w) for w in circ["wires"][g][:k]}


@pytest.mark.parametrize("make", [
    lambda: W.hea_circuit(20, 3, ring=True),
    lambda: W.hea_circuit(31, 2, ring=True),
    lambda: W.uccsd_instance(n=20, n_elec=10, n_singles=40, n_doubles=60, n_terms=30)["circuit"],
])
def test_fused_plan_keeps_dependencies_and_fits_tiles(make):
    """Host-side pass planner: a gate never moves ahead of an earlier gate it shares a qubit
    with, and every pass's non-diagonal gates act inside an 11-bit tile that keeps the low
    bits: 4 of them for HBM-resident states, 2 for states of at most 21 qubits (psi and lambda
    L2-resident)."""
    circ = make()
    low = set(range(2 if int(circ["n"]) <= 21 else 4))
    n_pass, pog = svqe.circuit_plan(circ)
    G = len(circ["types"])
    assert n_pass >= 1 and pog.min() == 0 and pog.max() == n_pass - 1
    for a in range(G):
        for b in range(a + 1, G):
            if _gate_bits(circ, a) & _gate_bits(circ, b):
                assert pog[a] <= pog[b], (a, b, pog[a], pog[b])
    for p in range(n_pass):
        bits = set()
        for g in np.flatnonzero(pog == p):
            if int(circ["types"][g]) != W.RZ:   # RZ runs are diagonal items: any bits
                bits |= _gate_bits(circ, g)
        assert len(bits | low) <= 11, (p, sorted(bits))
    # fusion actually fuses: far fewer passes than gates
    assert n_pass * 3 <= G


def test_layout_and_probe_calls_validate_their_arguments():
    """Host-side argument checks of the layout tuner's calls and the FP64 probe (no device
    work: every call below is rejected before a launch)."""
    for bad in ((0, 1, 2, 3), (13, 8, 2, 3), (10, 1, 2, 3), (12, 4, 2, 3), (5, 3, 2, 3),
                (5, 1, 0, 3), (5, 1, 2, 0)):
        with pytest.raises(svqe.SvError) as e:
            svqe.batch_set_layout(*bad)
        assert e.value.status == svqe.SV_EINVAL, bad
    svqe.batch_set_layout(9, 2, svqe.SEG_OFF, 3)  # valid: pinned, then forgotten
    svqe.batch_set_layout(9, 0, 0, 0)
    L = svqe.lib()
    assert L.sv_batch_layout(None, 5, None, None, None) == svqe.SV_EINVAL
    for shape in ((0, 128, 8, 10), (4, 100, 8, 10), (4, 2048, 8, 10), (4, 128, 3, 10),
                  (4, 128, 8, 0)):
        assert L.sv_fp64_probe(*shape, ctypes.c_void_p(16), None, None) == svqe.SV_EINVAL
    assert L.sv_fp64_probe(4, 128, 8, 10, None, None, None) == svqe.SV_EINVAL
