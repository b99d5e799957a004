"""torch.autograd wrapper: the misfit J(c) = 1/2 sum_s ||R u_s - d_s||^2 of the
Helmholtz solutions u_s = A(c)^{-1} f_s, differentiable with respect to the velocity c.

The forward pass sets up the sweeping preconditioner for c and calls hsweep_grad,
which solves the forward problems and the adjoint problems with the same
factorisation (A is complex symmetric) and forms dJ/dc in one fused kernel; the
backward pass scales that gradient by the incoming gradient.
"""
import torch

from . import default_opts, hsweep_setup


class HelmholtzMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, f, rec_idx, d, omega, pml_width, eps_H, tol, opts=None):
        h = hsweep_setup(c.detach(), omega, pml_width, eps_H, opts if opts is not None else default_opts())
        try:
            J, g = h.grad(f, rec_idx, d, tol)
        finally:
            h.free()
        ctx.save_for_backward(g.reshape(c.shape))
        return torch.tensor(J, dtype=torch.float64, device=c.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None, None, None, None, None


def helmholtz_misfit(c, f, rec_idx, d, omega, pml_width, eps_H=1e-6, tol=1e-8, opts=None):
    return HelmholtzMisfit.apply(c, f, rec_idx, d, omega, pml_width, eps_H, tol, opts)
