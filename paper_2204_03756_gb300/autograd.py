"""torch.autograd.Function over the hand-written adjoint of the MTPT run.

``mtpt_run(mass0, D, params, pos0, nsteps, checkpoint_every)`` advances the
particles ``nsteps`` time steps on the GPU and returns the final masses and
positions; ``backward`` runs the library's adjoint sweep (checkpointed
recomputation, binary64 adjoint passes) and returns dL/dM_0 and dL/dD.  The
gradient is pathwise: the walk's normals are fixed by the seed, bin and
pair-set changes contribute zero almost everywhere.  Every step, forward and
backward, runs in the CUDA library; this module only moves tensors.
"""
from __future__ import annotations

from dataclasses import replace

import torch

from . import mtpt


class _Run(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mass0, D, params, pos0, nsteps, checkpoint_every):
        p = replace(params, D=float(D.detach().cpu()))
        h = mtpt.mtpt_create(p)
        try:
            mtpt.mtpt_set_particles_device(h, p.dim, pos0.contiguous(),
                                           mass0.detach().contiguous())
            mtpt.mtpt_adjoint_forward(h, nsteps, checkpoint_every)
            n = mass0.numel()
            massT = torch.empty(n, dtype=torch.float64, device=mass0.device)
            posT = torch.empty(p.dim * n, dtype=torch.float64, device=mass0.device)
            mtpt.mtpt_get_masses_device(h, massT)
            mtpt.mtpt_get_positions_device(h, posT)
            mtpt.mtpt_sync(h)
        except Exception:
            mtpt.mtpt_destroy(h)
            raise
        ctx.h = h
        ctx.D_dtype = D.dtype
        ctx.D_device = D.device
        ctx.mark_non_differentiable(posT)
        return massT, posT.view(p.dim, n)

    @staticmethod
    def backward(ctx, g_massT, g_posT):
        h = ctx.h
        try:
            g = g_massT.contiguous().to(torch.float64)
            g0 = torch.empty_like(g)
            torch.cuda.current_stream().synchronize()
            dldD = mtpt.mtpt_adjoint_backward(h, g, g0)
        finally:
            mtpt.mtpt_destroy(h)
            ctx.h = None
        gD = torch.tensor(dldD, dtype=ctx.D_dtype, device=ctx.D_device)
        return g0, gD, None, None, None, None


def mtpt_run(mass0: torch.Tensor, D: torch.Tensor, params: mtpt.Params, pos0: torch.Tensor,
             nsteps: int, checkpoint_every: int = 20):
    """Final (masses, positions) after ``nsteps`` steps, differentiable in
    ``mass0`` (CUDA float64, n) and ``D`` (0-dim tensor)."""
    return _Run.apply(mass0, D, params, pos0, nsteps, checkpoint_every)


def binned_concentration(pos: torch.Tensor, mass: torch.Tensor, lo, hi, nbins):
    """C_b = sum of the masses in bin b / area of b, on an nbins[0] x nbins[1]
    grid over the box (bin membership is piecewise constant in the positions,
    so it carries no gradient)."""
    ix = ((pos[0] - lo[0]) / (hi[0] - lo[0]) * nbins[0]).long().clamp_(0, nbins[0] - 1)
    iy = ((pos[1] - lo[1]) / (hi[1] - lo[1]) * nbins[1]).long().clamp_(0, nbins[1] - 1)
    flat = ix * nbins[1] + iy
    area = (hi[0] - lo[0]) / nbins[0] * (hi[1] - lo[1]) / nbins[1]
    sums = torch.zeros(nbins[0] * nbins[1], dtype=mass.dtype, device=mass.device)
    sums = sums.index_add(0, flat, mass)
    return (sums / area).view(nbins[0], nbins[1])
