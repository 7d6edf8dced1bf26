"""The adjoint sweep behind torch.autograd.Function: its gradient against finite differences
(torch.autograd.gradcheck, float64) and against the oracle's parameter-shift gradient."""
import numpy as np
import pytest

import oracle
from paper_2601_09951_gb300 import svqe
from paper_2601_09951_gb300 import workloads as W
from tests.parity import assert_grad

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _setup(inst):
    from paper_2601_09951_gb300 import autograd as A
    stream = torch.cuda.current_stream().cuda_stream
    ctx = svqe.Context(inst["circuit"]["n"], stream=stream)
    ctx.init_reference(inst["ref"])
    H = svqe.Ham(ctx, inst["ham"])
    return A, ctx, H


@pytest.mark.parametrize("make", [
    lambda: W.hea_instance(6, 2, 40, 51, ring=True),
    lambda: W.uccsd_instance(n=8, n_elec=4, n_singles=5, n_doubles=5, n_terms=60, seed=52),
])
def test_gradcheck_and_parameter_shift(make):
    inst = make()
    A, ctx, H = _setup(inst)
    C = svqe.Circuit(inst["circuit"])
    theta = torch.tensor(inst["theta"], dtype=torch.float64, device="cuda", requires_grad=True)
    f = lambda t: A.vqe_energy(t, ctx, C, H)
    assert torch.autograd.gradcheck(f, (theta,), eps=1e-6, atol=1e-6, rtol=1e-5)
    e = f(theta)
    (g,) = torch.autograd.grad(3.0 * e, theta)
    _, g0 = oracle.energy_grad(inst)
    assert_grad(g.cpu().numpy() / 3.0, g0, inst["ham"])


def test_batch_energy_backward_weights_instances():
    from paper_2601_09951_gb300 import autograd as A
    insts = W.hea_batch(6)
    b = svqe.Batch(insts, stream=torch.cuda.current_stream().cuda_stream)
    theta = torch.tensor(b.theta_of(insts), device="cuda", requires_grad=True)
    w = torch.arange(1, 7, dtype=torch.float64, device="cuda")
    e = A.batch_energy(theta, b)
    (g,) = torch.autograd.grad((w * e).sum(), theta)
    g = g.cpu().numpy()
    for i, inst in enumerate(insts):
        _, g0 = oracle.energy_grad(inst)
        assert_grad(g[b.offsets[i]:b.offsets[i + 1]] / (i + 1), g0, inst["ham"])
