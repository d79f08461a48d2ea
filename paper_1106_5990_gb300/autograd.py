"""torch.autograd bridge of the reverse pass (amgd_backward).

``DistanceFn.apply(vals, omega, h, seed, nu, theta)`` runs the strength
build's forward path on handle ``h`` (values of A from the CUDA tensor
``vals``, start vectors from ``seed``, ``nu`` weighted-Jacobi sweeps with
weight ``omega``, distances for ``theta``) and returns the LS values per
slot of A (caller's slot order; NaN on the diagonal).  Its backward calls
amgd_backward with the incoming gradient as dL/dLS and returns dL/dvals and
dL/domega.  Every step runs in the library's kernels; torch only carries the
device memory.

``strength_loss(h, ...)`` is the built-in loss of the library (the sum of
r^2 = LS^-2 over the kept slots with LS > 0) with its gradient, as a
function of the same inputs; the library returns the loss and its gradient
from one call, so this function's forward already runs the reverse pass.
"""
from __future__ import annotations

import torch

from . import amgd


def _forward(h: amgd.Handle, vals, omega: float, seed: int, nu: int, theta: float,
             every: int):
    h.set_values(vals.detach().contiguous())
    h.set_checkpointing(every)
    h.init_vectors(seed)
    h.relax(nu, omega, amgd.AMGD_SWEEP_JACOBI)


class DistanceFn(torch.autograd.Function):
    """LS per slot as a differentiable function of A's values and omega."""

    @staticmethod
    def forward(ctx, vals, omega, h, seed, nu, theta, every=2):
        _forward(h, vals, float(omega), seed, nu, theta, every)
        ls = torch.empty(h.nnz, dtype=torch.float64, device=vals.device)
        h.distances(theta, want=("ls",), out={"ls": ls})
        ctx.h = h
        ctx.omega_device = omega.device if torch.is_tensor(omega) else None
        return ls

    @staticmethod
    def backward(ctx, g_ls):
        h = ctx.h
        g = torch.nan_to_num(g_ls.contiguous(), nan=0.0)
        vb = torch.empty_like(g)
        _, wb, _ = h.backward(ls_bar=g, out=vb)
        gw = (torch.tensor(wb, dtype=torch.float64, device=ctx.omega_device)
              if ctx.needs_input_grad[1] else None)
        return vb, gw, None, None, None, None, None


class StrengthLossFn(torch.autograd.Function):
    """The built-in loss sum r^2 over kept slots (flags held fixed)."""

    @staticmethod
    def forward(ctx, vals, omega, h, seed, nu, theta, every=2):
        _forward(h, vals, float(omega), seed, nu, theta, every)
        h.distances(theta, want=(), out={})
        vb = torch.empty(h.nnz, dtype=torch.float64, device=vals.device)
        _, wb, loss = h.backward(ls_bar=None, out=vb)
        ctx.save_for_backward(vb)
        ctx.wb = wb
        ctx.omega_device = omega.device if torch.is_tensor(omega) else None
        return torch.tensor(loss, dtype=torch.float64, device=vals.device)

    @staticmethod
    def backward(ctx, g):
        (vb,) = ctx.saved_tensors
        gw = None
        if ctx.needs_input_grad[1]:
            gw = ctx.wb * g.to(device=ctx.omega_device, dtype=torch.float64)
        return vb * g.to(vb.device), gw, None, None, None, None, None


def strength_loss(h, vals, omega, seed, nu, theta, every=2):
    return StrengthLossFn.apply(vals, omega, h, seed, nu, theta, every)
