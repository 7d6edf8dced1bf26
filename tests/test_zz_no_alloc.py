"""The no-device-allocation entry point (sv_adjoint_grad_noalloc), for callers that cannot
call cudaMalloc: they pass every buffer themselves and the library works in a fixed array of
its own.  Its energy and gradient must match the oracle and the ordinary entry point
(sv_adjoint_grad) within the parity tolerances, on two calls in a row (the shared array keeps
the first call's contents, which must not leak into the second), also when the caller writes
its inputs on a side stream and passes that stream.  Requests the array cannot hold, and
Hamiltonian records lowered for another register width, are rejected on the host; records
whose contents contradict the declared width or table size are caught on the device and give
NaN, with no read outside the buffers.  The buffers here are allocated by the test, playing
the caller's own memory."""
import numpy as np
import pytest

import oracle
from paper_2601_09951_gb300 import svqe
from paper_2601_09951_gb300 import workloads as W
from tests.parity import assert_energy, assert_grad

pytestmark = pytest.mark.gpu


def _device(torch, arr, dtype):
    return torch.from_numpy(np.ascontiguousarray(arr).view(dtype)).to("cuda")


def _noalloc(torch, inst, theta, stream=None, ham=None, ham_n=None, lower_n=None,
             n_table=None):
    """One call with buffers made on `stream` (torch's current stream if None); the records
    are lowered for lower_n qubits and declared as ham_n-qubit records (both default to the
    circuit's width)."""
    n = inst["circuit"]["n"]
    ham_n = n if ham_n is None else ham_n
    lower_n = ham_n if lower_n is None else lower_n
    rec, table = svqe.group_records(inst["ham"] if ham is None else ham, lower_n)
    s = torch.cuda.current_stream() if stream is None else stream
    with torch.cuda.stream(s):
        g_d = _device(torch, rec.view(np.uint8), np.uint8)
        t_d = _device(torch, table.view(np.float64), np.float64)
        th_d = torch.tensor(theta, dtype=torch.float64, device="cuda")
        e_d = torch.zeros(1, dtype=torch.float64, device="cuda")
        gr_d = torch.zeros(max(len(theta), 1), dtype=torch.float64, device="cuda")
        svqe.adjoint_grad_noalloc(inst["circuit"], inst["ref"], ham_n, g_d.data_ptr(), len(rec),
                                  t_d.data_ptr(), len(table) if n_table is None else n_table,
                                  th_d.data_ptr(), e_d.data_ptr(), gr_d.data_ptr(),
                                  s.cuda_stream)
    s.synchronize()
    return float(e_d.item()), gr_d.cpu().numpy()[:len(theta)]


def _ordinary(inst, theta):
    n = inst["circuit"]["n"]
    ctx = svqe.Context(n)
    ctx.init_reference(inst["ref"])
    H = svqe.Ham(ctx, inst["ham"])
    return ctx.adjoint_grad(inst["circuit"], theta, H)


MAKERS = [
    lambda: W.hea_instance(8, 3, 120, 21, ring=True),
    lambda: W.h2_sweep(100)[55],
    lambda: W.uccsd_instance(n=10, n_elec=4, n_singles=10, n_doubles=14, n_terms=160, seed=8),
]


@pytest.mark.parametrize("make", MAKERS)
def test_two_calls_in_a_row_match_the_ordinary_entry_point_and_the_oracle(make):
    torch = pytest.importorskip("torch")
    inst = make()
    rng = np.random.default_rng(3)
    thetas = [np.asarray(inst["theta"], np.float64),
              rng.uniform(-np.pi, np.pi, size=len(inst["theta"]))]
    for theta in thetas:
        e, g = _noalloc(torch, inst, theta)
        e0, g0 = _ordinary(inst, theta)
        assert_energy(e, e0, inst["ham"], "no-alloc vs sv_adjoint_grad")
        assert_grad(g, g0, inst["ham"], "no-alloc vs sv_adjoint_grad")
        eo, go = oracle.energy_grad(inst, theta)
        assert_energy(e, eo, inst["ham"], "no-alloc vs oracle")
        assert_grad(g, go, inst["ham"], "no-alloc vs oracle")


def test_inputs_written_on_a_side_stream():
    torch = pytest.importorskip("torch")
    inst = MAKERS[0]()
    side = torch.cuda.Stream()
    for theta in (np.asarray(inst["theta"], np.float64), -np.asarray(inst["theta"], np.float64)):
        e, g = _noalloc(torch, inst, theta, stream=side)
        eo, go = oracle.energy_grad(inst, theta)
        assert_energy(e, eo, inst["ham"], "side stream")
        assert_grad(g, go, inst["ham"], "side stream")


def test_requests_beyond_the_array_are_rejected():
    torch = pytest.importorskip("torch")
    big = W.hea_instance(svqe.NOALLOC_MAX_QUBITS + 1, 1, 10, 1)
    with pytest.raises(svqe.SvError) as e:
        _noalloc(torch, big, big["theta"])
    assert e.value.status == svqe.SV_EINVAL and "qubits" in str(e.value)
    long = W.hea_instance(6, 30, 10, 1)  # 30 layers x 17 gates > 256 gates
    with pytest.raises(svqe.SvError) as e:
        _noalloc(torch, long, long["theta"])
    assert e.value.status == svqe.SV_EINVAL and "gates" in str(e.value)


def test_records_for_another_register_width_are_rejected_on_the_host():
    torch = pytest.importorskip("torch")
    inst = W.hea_instance(6, 2, 40, 5)
    wide = W.hea_instance(8, 2, 40, 5)["ham"]
    with pytest.raises(svqe.SvError) as e:
        _noalloc(torch, inst, inst["theta"], ham=wide, ham_n=8)
    assert e.value.status == svqe.SV_EINVAL and "qubits" in str(e.value)
    with pytest.raises(svqe.SvError) as e:
        _noalloc(torch, inst, inst["theta"], n_table=0)
    assert e.value.status == svqe.SV_EINVAL


def test_records_that_contradict_the_declared_width_give_nan_then_recover():
    """Records lowered for 8 qubits (mask bits 6 and 7 set) but declared as 6-qubit records,
    and a declared table smaller than the records' ranges, are caught by the device-side check:
    the outputs are NaN and nothing outside the buffers is read.  The next valid call on the
    same array is exact again."""
    torch = pytest.importorskip("torch")
    inst = W.hea_instance(6, 2, 40, 5)
    wide = W.hea_instance(8, 2, 40, 5)["ham"]
    rec, _ = svqe.group_records(wide, 8)
    assert np.any((rec["x_mask"] | rec["z_union"]) >> np.uint64(6))
    e, g = _noalloc(torch, inst, inst["theta"], ham=wide, ham_n=6, lower_n=8)
    assert np.isnan(e) and np.all(np.isnan(g))
    e, g = _noalloc(torch, inst, inst["theta"], n_table=1)
    assert np.isnan(e) and np.all(np.isnan(g))
    e, g = _noalloc(torch, inst, inst["theta"])
    eo, go = oracle.energy_grad(inst)
    assert_energy(e, eo, inst["ham"], "after a rejected call")
    assert_grad(g, go, inst["ham"], "after a rejected call")
