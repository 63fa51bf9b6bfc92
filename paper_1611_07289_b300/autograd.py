"""Differentiable forward model: simulate_patches as a torch.autograd.Function.

Forward: pvr_simulate (Eq. 1, the Gaussian-PSF forward model of every patch
at its pose).  Backward, for an upstream gradient g = dL/dsim:

* dL/dx     = A^T g over the valid pixels      (pvr_adjoint, the K4 kernel)
* dL/dposes = sum_pix g_pix d sim_pix / d pose  (pvr_pose_grad)

Both backward kernels recompute the PSF weights and sample positions from
the poses; the forward pass stores nothing but its inputs.  Invalid pixels
(no in-volume PSF weight) are constant zeros of the forward model, so their
upstream gradient is ignored.  The derivative holds the PSF normalisation
constant, as the registration gradient does (it changes only where a sample
leaves the volume).

This module only marshals arguments; every step runs in libpvr's kernels.
"""
from __future__ import annotations

import torch

from . import pvr as _pvr


class SimulatePatches(torch.autograd.Function):
    """sim, valid = SimulatePatches.apply(x, poses, ctx, patch_table)

    x: float32 volume [nz, ny, nx] on the GPU; poses: float64 [n, n_params]
    (6 rigid or 12 affine, as the context);
    ctx: pvr.Context; patch_table: pvr.PatchTable.  sim: float32 [n_pix];
    valid: uint8 [n_pix] (not differentiable)."""

    @staticmethod
    def forward(fctx, x, poses, ctx: "_pvr.Context", pt: "_pvr.PatchTable"):
        x_c, p_c = x.detach().contiguous(), poses.detach().contiguous()
        sim, valid = ctx.pvr_simulate(x_c, pt, p_c)
        fctx.save_for_backward(x_c, p_c)
        fctx.pvr_ctx, fctx.pt = ctx, pt
        fctx.mark_non_differentiable(valid)
        return sim, valid

    @staticmethod
    def backward(fctx, g_sim, g_valid):
        x, poses = fctx.saved_tensors
        ctx, pt = fctx.pvr_ctx, fctx.pt
        g = g_sim.detach().to(torch.float32).contiguous()
        gx = gp = None
        if fctx.needs_input_grad[0]:
            gx, _ = ctx.pvr_adjoint(pt, poses, r=g, w=None)
            gx = gx.reshape(x.shape)
        if fctx.needs_input_grad[1]:
            gp = ctx.pvr_pose_grad(x, g, pt, poses)
        return gx, gp, None, None


def simulate_patches(x, poses, ctx, pt):
    """Differentiable forward model; returns (sim, valid)."""
    return SimulatePatches.apply(x, poses, ctx, pt)
