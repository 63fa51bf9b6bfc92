"""Training and use of the learned pose proposal (pvr_net).

Training pairs are made by the forward model itself: for a phantom volume x
and a 64x64 patch at its acquired position, the "acquired" patch is
y = simulate(x, 0) and the network input is (y, simulate(x, delta)) for a
random rigid perturbation drawn in the frame of the patch's stack
(translations up to +-trans mm along, rotations up to +-rot degrees about
its unit column, row and normal directions; in world pose parameters
delta = (S t, S w) with S those unit axes); the target is the correction
-(t, w), divided by SCALE so that it is of order one.  The stack frame
makes the target a function of the two images alone (an image shift means
the same frame translation for every stack orientation).  In use,
pvr_pose_propose maps the predicted correction to world parameters with the
same S, applies it where it raises NCC and keeps the plain pose elsewhere;
NCC registration then refines.

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


def stack_axes(geom, desc):
    """Per patch, the 3x3 matrix S whose columns are the unit column, row and
    slice-normal directions of the patch's stack (float64 [n, 3, 3])."""
    P = np.stack([np.asarray(geom.p2w[s], np.float64)[:, :3] for s in range(len(geom.p2w))])
    P = P / np.linalg.norm(P, axis=1, keepdims=True)
    return P[np.asarray(desc[:, 0])]


def frame_to_world(S, local):
    """World pose increments (S t, S w) of stack-frame corrections (t, w)."""
    return np.concatenate([np.einsum("nij,nj->ni", S, local[:, :3]), np.einsum("nij,nj->ni", S, local[:, 3:])], 1)


def phantom_volumes(geom, seeds, device="cuda"):
    """Random uterus phantoms (synth.phantom_uterus) at the voxel centres."""
    vols = []
    for sd in seeds:
        ells, _ = synth.phantom_uterus(np.random.default_rng(int(sd)))
        vols.append(synth.ground_truth(ells, geom, device=device).to(device).contiguous())
    return vols


def train(net: "_pvr.Net", ctx: "_pvr.Context", vols, pt: "_pvr.PatchTable", n_pairs, batch=256, lr=1e-3,
          rot=20.0, trans=10.0, seed=0, log=None, geom=None):
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
    S_all = stack_axes(geom, pt.desc.cpu().numpy())
    for it in range(steps):
        v = int(rng.integers(len(vols)))
        rows_np = rng.choice(pt.n, batch, replace=False)
        rows = torch.as_tensor(rows_np, device=dev)
        sub = _pvr.PatchTable(pt.desc[rows].contiguous(), n_pix, 64)
        local = np.concatenate([rng.uniform(-trans, trans, (batch, 3)), rng.uniform(-rot, rot, (batch, 3))], 1)
        delta = torch.as_tensor(frame_to_world(S_all[rows_np], local), device=dev)
        ctx.pvr_simulate(vols[v], sub, delta, s, valid)
        target = (-torch.as_tensor(local, device=dev) / scale).to(torch.float32).contiguous()
        net.train_step(ys[v], s, valid, sub, 0, batch, target, lr * (0.5 ** (3 * it / steps)), loss)
        if it % 50 == 0 or it == steps - 1:
            losses.append((it, float(loss)))
            if log:
                log(f"step {it}/{steps} loss {losses[-1][1]:.4f}")
    torch.cuda.synchronize()
    return losses, time.perf_counter() - t0


def evaluate_proposal(net: "_pvr.Net", ctx: "_pvr.Context", x, pt: "_pvr.PatchTable", n, rot=10.0, trans=5.0,
                      seed=1, geom=None):
    """Mean absolute pose error (mm, degrees; world parameters) of n random
    perturbed patches (drawn in the stack frame, as in training) before and
    after one proposal on the clean volume x, and the fraction of proposals
    taken."""
    dev = pt.desc.device
    rng = np.random.default_rng(seed)
    rows = torch.as_tensor(rng.choice(pt.n, n, replace=False), device=dev)
    sub = _pvr.PatchTable(pt.desc[rows].contiguous(), pt.n_pix, 64)
    zeros = torch.zeros((n, 6), dtype=torch.float64, device=dev)
    y = torch.zeros(pt.n_pix, dtype=torch.float32, device=dev)
    v = torch.zeros(pt.n_pix, dtype=torch.uint8, device=dev)
    ctx.pvr_simulate(x, sub, zeros, y, v)
    local = np.concatenate([rng.uniform(-trans, trans, (n, 3)), rng.uniform(-rot, rot, (n, 3))], 1)
    delta = torch.as_tensor(frame_to_world(stack_axes(geom, pt.desc[rows].cpu().numpy()), local), device=dev)
    poses = delta.clone()
    acc = torch.zeros(n, dtype=torch.int32, device=dev)
    net.propose(ctx, x, y, sub, poses, SCALE, acc)
    before = delta.abs().mean(0).cpu().numpy()
    after = poses.abs().mean(0).cpu().numpy()
    return before, after, float(acc.float().mean())
