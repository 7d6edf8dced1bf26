"""Host logic of the batched kernel's segmentation (sv_batch_segments, no device work): the
invariants the kernel relies on.  Segments tile the gate list in order; every kind holds only
the gates it may hold, within the kernel's fixed capacities (16 RZ and 16 CZ per diagonal run,
2..32 CNOT/X per permutation run, at most 16 distinct-qubit rotations per layer); checkpoint
slots, which also index a fused segment's saved tables, are numbered 0, 1, ... in forward order
and are absent only where the kernel takes none."""
import ctypes

import numpy as np
import pytest

from paper_2601_09951_gb300 import svqe
from paper_2601_09951_gb300 import workloads as W

GATES, RLAYER, DIAG, PERM, DIAGPERM = 0, 1, 2, 3, 4
AUX_AMPS = 176  # amplitudes of saved tables per checkpoint slot


def _circuit(n, gates):
    cb = W.CircuitBuilder(n)
    for g, wires in gates:
        cb.add(g, wires, param="new" if g in (W.RX, W.RY, W.RZ) else None)
    return cb.build()


def _check_invariants(circ):
    segs, n_ckpt, scratch = svqe.batch_segments(circ)
    types = np.asarray(circ["types"])
    wires = np.asarray(circ["wires"])
    # segments tile [0, n_gates) in order
    pos = 0
    for kind, split, first, count, ck in segs:
        assert first == pos and count > 0
        pos += count
    assert pos == len(types)
    # checkpoint slots 0..n_ckpt-1 in order, -1 only for plain gates and a product layer
    slots = [int(s[4]) for s in segs if s[4] >= 0]
    assert slots == list(range(n_ckpt))
    for i, (kind, split, first, count, ck) in enumerate(segs):
        t = types[first:first + count]
        if kind == GATES:
            assert ck == -1
        elif kind == RLAYER:
            assert 2 <= count <= 16
            assert len(set(t.tolist())) == 1 and t[0] in (W.RY, W.RX)
            q = wires[first:first + count, 0]
            assert len(set(q.tolist())) == count
            if split == 1:
                assert i == 0 and first == 0 and t[0] == W.RY and ck == -1
            else:
                assert split == 0 and ck >= 0
        elif kind in (DIAG, DIAGPERM):
            nd = count if kind == DIAG else split
            d = t[:nd]
            assert set(d.tolist()) <= {W.RZ, W.CZ}
            assert 3 <= int(np.sum(d == W.RZ)) <= 16 and int(np.sum(d == W.CZ)) <= 16
            if kind == DIAGPERM:
                p = t[nd:]
                assert 2 <= len(p) <= 32 and set(p.tolist()) <= {W.CNOT, W.X}
            assert ck >= 0
        elif kind == PERM:
            assert 2 <= count <= 32 and set(t.tolist()) <= {W.CNOT, W.X} and ck >= 0
        else:
            raise AssertionError(f"unknown segment kind {kind}")
    assert scratch == n_ckpt * ((1 << circ["n"]) + AUX_AMPS)
    return segs, n_ckpt


@pytest.mark.parametrize("i", range(0, 64, 3))
def test_batched_workload_segments(i):
    """Hardware-efficient instances: a product first layer, then (diagonal + CNOT ladder,
    commuting layer) pairs, and a final diagonal + ladder segment."""
    inst = W.hea_batch(64)[i]
    circ = inst["circuit"]
    segs, n_ckpt = _check_invariants(circ)
    n = circ["n"]
    L = len(segs) // 2
    kinds = [int(s[0]) for s in segs]
    assert kinds == [RLAYER] + [DIAGPERM, RLAYER] * (L - 1) + [DIAGPERM]
    assert segs[0][1] == 1 and segs[0][3] == n
    assert n_ckpt == len(segs) - 1


def test_long_runs_are_cut_at_the_kernel_capacities():
    n = 12
    gates = [(W.RY, [q]) for q in range(n)]            # product layer
    gates += [(W.RZ, [q % n]) for q in range(20)]       # 20 RZ: 16, then 4
    gates += [(W.CNOT, [q % n, (q + 1) % n]) for q in range(40)]  # 40 CNOT: 32, then 8
    gates += [(W.RX, [q]) for q in range(5)] + [(W.RX, [2])]      # repeat ends the layer
    circ = _circuit(n, gates)
    segs, _ = _check_invariants(circ)
    kinds = [(int(k), int(c)) for k, _, _, c, _ in segs]
    assert kinds[0] == (RLAYER, 12)
    assert kinds[1] == (DIAG, 16)
    assert kinds[2] == (DIAGPERM, 4 + 32)
    assert kinds[3] == (PERM, 8)
    assert kinds[4] == (RLAYER, 5)
    assert kinds[5] == (GATES, 1)


def test_short_runs_stay_plain_gates():
    n = 6
    gates = [(W.RX, [0]), (W.RZ, [1]), (W.RZ, [2]), (W.CNOT, [0, 1]), (W.H, [3]),
             (W.RY, [4]), (W.CZ, [1, 2])]
    segs, n_ckpt = _check_invariants(_circuit(n, gates))
    assert [int(s[0]) for s in segs] == [GATES]
    assert n_ckpt == 0


def test_first_rx_layer_is_not_a_product_layer():
    n = 5
    gates = [(W.RX, [q]) for q in range(n)] + [(W.RY, [q]) for q in range(n)]
    segs, n_ckpt = _check_invariants(_circuit(n, gates))
    assert [(int(s[0]), int(s[1])) for s in segs] == [(RLAYER, 0), (RLAYER, 0)]
    assert n_ckpt == 2


def test_empty_circuit_and_small_capacity():
    segs, n_ckpt, scratch = svqe.batch_segments(_circuit(3, []))
    assert len(segs) == 0 and n_ckpt == 0 and scratch == 0
    circ = W.hea_batch(1)[0]["circuit"]
    C = svqe.Circuit(circ)
    ns, nc = ctypes.c_int32(), ctypes.c_int32()
    buf = np.zeros((1, 5), np.int32)
    st = svqe.lib().sv_batch_segments(C.ref(), 1, buf.ctypes.data, ctypes.byref(ns),
                                      ctypes.byref(nc), None)
    assert st == 1  # SV_EINVAL: more segments than rows
    # NULL circuit or outputs: SV_EINVAL, nothing written
    assert svqe.lib().sv_batch_segments(None, 0, None, ctypes.byref(ns), ctypes.byref(nc),
                                        None) == 1
    assert svqe.lib().sv_batch_segments(C.ref(), 0, None, None, None, None) == 1
