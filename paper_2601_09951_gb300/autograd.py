"""torch.autograd.Function wrappers of the adjoint sweep.

The energy E(theta) = <ref|U(theta)^dag H U(theta)|ref> (Sec. 3.1, Eq. 2) and its gradient
come from one call of the library's adjoint path (sv_adjoint_grad_dev / sv_batch_run_dev):
forward pass, lambda = H psi, reverse sweep.  The forward of these Functions runs that call and
keeps the gradient; their backward multiplies it by the incoming gradient.  PyTorch supplies
the device buffers and the stream; the arithmetic is the library's.
"""
import torch

from . import svqe


def _check_theta(theta):
    if theta.dtype != torch.float64 or not theta.is_cuda or theta.dim() != 1:
        raise TypeError("theta must be a 1-D float64 CUDA tensor")
    return theta.contiguous()


class VQEEnergy(torch.autograd.Function):
    """E(theta) of one state; `context` must order its work on torch's current stream (create
    it with stream=torch.cuda.current_stream().cuda_stream)."""

    @staticmethod
    def forward(ctx, theta, context, circuit, ham):
        theta = _check_theta(theta)
        e = torch.empty(1, dtype=torch.float64, device=theta.device)
        g = torch.empty_like(theta)
        context.adjoint_grad_dev(circuit, theta.data_ptr(), ham, e.data_ptr(), g.data_ptr())
        ctx.save_for_backward(g)
        return e[0]

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None


class BatchEnergy(torch.autograd.Function):
    """Energies of every instance of an svqe.Batch (created on torch's current stream), with
    theta the concatenated parameters."""

    @staticmethod
    def forward(ctx, theta, batch):
        theta = _check_theta(theta)
        e = torch.empty(batch.n_instances, dtype=torch.float64, device=theta.device)
        g = torch.empty_like(theta)
        batch.run_dev(theta.data_ptr(), e.data_ptr(), g.data_ptr())
        ctx.save_for_backward(g)
        ctx.counts = torch.as_tensor(batch.offsets[1:] - batch.offsets[:-1],
                                     device=theta.device)
        return e

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        scale = torch.repeat_interleave(grad_out, ctx.counts)
        return scale * g, None


def vqe_energy(theta, context, circuit, ham):
    C = circuit if isinstance(circuit, svqe.Circuit) else svqe.Circuit(circuit)
    return VQEEnergy.apply(theta, context, C, ham)


def batch_energy(theta, batch):
    return BatchEnergy.apply(theta, batch)
