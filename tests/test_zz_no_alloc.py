"""The no-device-allocation entry point (sv_adjoint_grad_noalloc), for callers that cannot
call cudaMalloc: they pass every buffer themselves and the library works in a fixed array of
its own.  Its energy and gradient must match the ordinary entry point's (sv_adjoint_grad)
within the parity tolerances, on two calls in a row (the shared array keeps the first call's
contents, which must not leak into the second).  The buffers here are allocated by the test,
playing the caller's own memory."""
import numpy as np
import pytest

from paper_2601_09951_gb300 import svqe
from paper_2601_09951_gb300 import workloads as W
from tests.parity import assert_energy, assert_grad

pytestmark = pytest.mark.gpu


def _device(torch, arr, dtype):
    return torch.from_numpy(np.ascontiguousarray(arr).view(dtype)).to("cuda")


def _noalloc(torch, inst, theta):
    n = inst["circuit"]["n"]
    rec, table = svqe.group_records(inst["ham"], n)
    g_d = _device(torch, rec.view(np.uint8), np.uint8)
    t_d = _device(torch, table.view(np.float64), np.float64)
    th_d = torch.tensor(theta, dtype=torch.float64, device="cuda")
    e_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    gr_d = torch.zeros(max(len(theta), 1), dtype=torch.float64, device="cuda")
    svqe.adjoint_grad_noalloc(inst["circuit"], inst["ref"], g_d.data_ptr(), len(rec),
                              t_d.data_ptr(), th_d.data_ptr(), e_d.data_ptr(), gr_d.data_ptr())
    torch.cuda.synchronize()
    return float(e_d.item()), gr_d.cpu().numpy()[:len(theta)]


def _ordinary(inst, theta):
    n = inst["circuit"]["n"]
    ctx = svqe.Context(n)
    ctx.init_reference(inst["ref"])
    H = svqe.Ham(ctx, inst["ham"])
    return ctx.adjoint_grad(inst["circuit"], theta, H)


@pytest.mark.parametrize("make", [
    lambda: W.hea_instance(8, 3, 120, 21, ring=True),
    lambda: W.h2_sweep(100)[55],
    lambda: W.uccsd_instance(n=10, n_elec=4, n_singles=10, n_doubles=14, n_terms=160, seed=8),
])
def test_two_calls_in_a_row_match_the_ordinary_entry_point(make):
    torch = pytest.importorskip("torch")
    inst = make()
    rng = np.random.default_rng(3)
    thetas = [np.asarray(inst["theta"], np.float64),
              rng.uniform(-np.pi, np.pi, size=len(inst["theta"]))]
    for theta in thetas:
        e, g = _noalloc(torch, inst, theta)
        e0, g0 = _ordinary(inst, theta)
        assert_energy(e, e0, inst["ham"], "no-alloc")
        assert_grad(g, g0, inst["ham"], "no-alloc")


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
