"""torch.autograd front end of the open-GRAPE gradient.

``GrapeFunction.apply(u, problem)`` returns Phi(u) as a 0-dim tensor whose
backward pass yields dPhi/du from the library's adjoint sweep (exact
derivative of the RK4 map, or the paper's first-order Eq. (dphidu), as the
problem was created).  Long pulses are handled inside the library by
checkpoint segments: states are kept every ``ckpt_stride`` slices and each
segment's stage inputs are recomputed before its adjoint sweep, so memory
grows with N_t / stride + stride instead of N_t.

Two evaluation strategies:
  fused=True   forward runs the whole gradient evaluation and keeps dPhi/du
               (one forward and one adjoint sweep when backward follows);
  fused=False  forward propagates only; backward runs the gradient
               evaluation (cheaper when backward is usually skipped).
All arithmetic runs in libgrape.so; torch provides the tensors and streams.
"""
from __future__ import annotations

import torch

from . import _lib


class GrapeFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, problem, fused=True):
        if not (u.is_cuda and u.dtype == torch.float64):
            raise TypeError("u must be a float64 CUDA tensor of shape (n_slices, n_controls)")
        u = u.contiguous()
        stream = torch.cuda.current_stream(u.device)
        if fused:
            F, G = problem.gradient(u, stream=stream)
            ctx.save_for_backward(G)
        else:
            F, _ = problem.forward(u, stream=stream, want_rho=False)
            ctx.save_for_backward(u)
        ctx.problem = problem
        ctx.fused = fused
        return F.reshape(())

    @staticmethod
    def backward(ctx, gF):
        (saved,) = ctx.saved_tensors
        if ctx.fused:
            G = saved
        else:
            _, G = ctx.problem.gradient(saved, stream=torch.cuda.current_stream(saved.device))
        return gF * G, None, None


def grape_phi(u, problem, fused=True):
    """Phi(u) with autograd support (see GrapeFunction)."""
    return GrapeFunction.apply(u, problem, fused)


class FilterFunction(torch.autograd.Function):
    """s = T u for a GaussianFilter (App. A); backward applies the transposed
    filter, the chain rule of the paper's filtered gradient."""

    @staticmethod
    def forward(ctx, u, filt):
        if not (u.is_cuda and u.dtype == torch.float64):
            raise TypeError("u must be a float64 CUDA tensor of shape (n_steps, n_controls)")
        ctx.filt = filt
        return filt.apply(u, stream=torch.cuda.current_stream(u.device))

    @staticmethod
    def backward(ctx, g_s):
        return ctx.filt.adjoint(g_s, stream=torch.cuda.current_stream(g_s.device)), None


def gaussian_filter(u, filt):
    """Differentiable Gaussian filtering of the controls u (n_steps x R)."""
    return FilterFunction.apply(u, filt)
