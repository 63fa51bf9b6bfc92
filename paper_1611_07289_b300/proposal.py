"""Training and use of the learned pose proposal (pvr_net).

Training pairs are made by the forward model itself: for a phantom volume x
and a 64x64 patch at its acquired position, the "acquired" patch is
y = simulate(x, 0) and the network input is (y, simulate(x, delta)) for a
random rigid perturbation delta (rotations up to +-rot degrees,
translations up to +-trans mm); the target is the correction -delta,
divided by SCALE so that it is of order one.  In use, pvr_pose_propose
applies the predicted correction where it raises NCC and keeps the plain
pose elsewhere; NCC registration then refines.

This module only chooses batches and marshals arguments; every step runs in
libpvr (pvr_simulate, pvr_net_train_step, pvr_pose_propose).
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import pvr as _pvr
from . import synth

SCALE = (10.0, 10.0, 10.0, 20.0, 20.0, 20.0)   # mm, mm, mm, degrees, degrees, degrees


def phantom_volumes(geom, seeds, device="cuda"):
    """Random uterus phantoms (synth.phantom_uterus) at the voxel centres."""
    vols = []
    for sd in seeds:
        ells, _ = synth.phantom_uterus(np.random.default_rng(int(sd)))
        vols.append(synth.ground_truth(ells, geom, device=device).to(device).contiguous())
    return vols


def train(net: "_pvr.Net", ctx: "_pvr.Context", vols, pt: "_pvr.PatchTable", n_pairs, batch=256, lr=1e-3,
          rot=20.0, trans=10.0, seed=0, log=None):
    """Train on n_pairs perturbed patches drawn from the table over the given
    volumes; returns the list of batch losses and the wall time."""
    dev = pt.desc.device
    rng = np.random.default_rng(seed)
    n_pix = pt.n_pix
    zeros = torch.zeros((pt.n, 6), dtype=torch.float64, device=dev)
    ys = [ctx.pvr_simulate(x, pt, zeros)[0] for x in vols]
    s = torch.zeros(n_pix, dtype=torch.float32, device=dev)
    valid = torch.zeros(n_pix, dtype=torch.uint8, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    scale = torch.tensor(SCALE, dtype=torch.float64, device=dev)
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps = max(1, n_pairs // batch)
    for it in range(steps):
        v = int(rng.integers(len(vols)))
        rows = torch.as_tensor(rng.choice(pt.n, batch, replace=False), device=dev)
        sub = _pvr.PatchTable(pt.desc[rows].contiguous(), n_pix, 64)
        delta = torch.as_tensor(np.concatenate([rng.uniform(-trans, trans, (batch, 3)),
                                                rng.uniform(-rot, rot, (batch, 3))], 1), device=dev)
        ctx.pvr_simulate(vols[v], sub, delta, s, valid)
        target = (-delta / scale).to(torch.float32).contiguous()
        net.train_step(ys[v], s, valid, sub, 0, batch, target, lr * (0.5 ** (3 * it / steps)), loss)
        if it % 50 == 0 or it == steps - 1:
            losses.append((it, float(loss)))
            if log:
                log(f"step {it}/{steps} loss {losses[-1][1]:.4f}")
    torch.cuda.synchronize()
    return losses, time.perf_counter() - t0


def evaluate_proposal(net: "_pvr.Net", ctx: "_pvr.Context", x, pt: "_pvr.PatchTable", n, rot=10.0, trans=5.0,
                      seed=1):
    """Mean absolute pose error (mm, degrees) of n random perturbed patches
    before and after one proposal on the clean volume x, and the fraction of
    proposals taken."""
    dev = pt.desc.device
    rng = np.random.default_rng(seed)
    rows = torch.as_tensor(rng.choice(pt.n, n, replace=False), device=dev)
    sub = _pvr.PatchTable(pt.desc[rows].contiguous(), pt.n_pix, 64)
    zeros = torch.zeros((n, 6), dtype=torch.float64, device=dev)
    y = torch.zeros(pt.n_pix, dtype=torch.float32, device=dev)
    v = torch.zeros(pt.n_pix, dtype=torch.uint8, device=dev)
    ctx.pvr_simulate(x, sub, zeros, y, v)
    delta = torch.as_tensor(np.concatenate([rng.uniform(-trans, trans, (n, 3)), rng.uniform(-rot, rot, (n, 3))], 1),
                            device=dev)
    poses = delta.clone()
    acc = torch.zeros(n, dtype=torch.int32, device=dev)
    net.propose(ctx, x, y, sub, poses, SCALE, acc)
    before = delta.abs().mean(0).cpu().numpy()
    after = poses.abs().mean(0).cpu().numpy()
    return before, after, float(acc.float().mean())
