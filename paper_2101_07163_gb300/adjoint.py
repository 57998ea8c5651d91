"""Differentiable rollout of the ice-growth solver for PyTorch autograd.

``rollout(phi0, U0, eps, D, nsteps=...)`` advances a grid from the equilibrium state of the
moment fields (phi0, U0; fluid at rest) and returns phi after nsteps steps. Its backward is
the discrete adjoint of the step on the GPU (include/lbmice.h, lbmice_tape_*): checkpoints
every ``every`` steps, each segment recomputed and swept backwards. This module only moves
arguments between PyTorch and the C ABI; every forward and reverse step runs in the CUDA
kernels of liblbmice.so.
"""
from __future__ import annotations

import torch

from . import lbmice


class Rollout(torch.autograd.Function):
    """phi_T = Rollout.apply(phi0, U0, eps, D, spec). phi0: (ny, nx) CUDA tensor; U0: a
    0-dim tensor (uniform supersaturation) or a (ny, nx) field; eps, D: 0-dim tensors;
    spec: dict with nsteps, every and further make_params keywords (periodic faces,
    FP32 storage). Gradients flow to all four tensors; D includes its effect through the
    beta = 0 lambda unless spec gives lam."""

    @staticmethod
    def forward(ctx, phi0, U0, eps, D, spec):
        spec = dict(spec)
        nsteps, every = int(spec.pop("nsteps")), int(spec.pop("every", 100))
        ny, nx = phi0.shape
        lat = lbmice.Lattice(nx, ny, eps=float(eps), D=float(D), **spec)
        Uf = U0.expand(ny, nx) if U0.dim() == 0 else U0
        lat.set_fields(phi=phi0.detach().to(torch.float64), U=Uf.detach().to(torch.float64))
        tape = lbmice.Tape(lat, every)
        tape.record(nsteps)
        out = torch.empty((ny, nx), dtype=torch.float32, device=phi0.device)
        lat.field(lbmice.PHI, out=out)
        ctx.lat, ctx.tape = lat, tape
        ctx.meta = (phi0.dtype, U0.dim() == 0, U0.dtype, eps.dtype, D.dtype)
        return out

    @staticmethod
    def backward(ctx, g):
        # The tape may be swept again (backward with retain_graph=True, then another
        # backward); its checkpoints and the grid are freed with the autograd graph that
        # holds ctx.
        dphi, scalar_U, dU, deps, dD = ctx.meta
        grads, fields = ctx.tape.backward(phi_bar=g.detach().contiguous())
        gU = fields["U0"].sum() if scalar_U else fields["U0"]
        dev = g.device
        return (fields["phi0"].to(dphi), gU.to(dU),
                torch.tensor(grads["eps"], dtype=deps, device=dev),
                torch.tensor(grads["D"], dtype=dD, device=dev), None)


def rollout(phi0, U0, eps, D, *, nsteps: int, every: int = 100, **params):
    """phi after ``nsteps`` steps, differentiable in phi0, U0, eps and D."""
    return Rollout.apply(phi0, U0, eps, D, dict(nsteps=nsteps, every=every, **params))
