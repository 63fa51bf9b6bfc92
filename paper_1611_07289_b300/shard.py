"""Host logic of the patch-sharded form of one reconstruction pass.

Patches are independent given the volume (Sec. II-D: every patch is
simulated, weighted and registered on its own), so one reconstruction
problem splits over R ranks as follows:

* every rank holds a replica of the volume x and the EM state;
* the patch table is cut into R contiguous row ranges with balanced pixel
  counts (``partition_by_pixels``); each rank's rows are rebased so its
  patch pixels start at offset 0 (``shard_table``);
* the forward model, residuals, per-patch potentials and registration run on
  each rank's own rows with no exchange;
* the exchanges per super-resolution pass are the global EM sums: before
  the E-step the pixel count, sum e^2 and max / min of e (the first call's
  sigma^2 and the outlier density m, ``em_global_stats``), after it sum p and
  sum p e^2 (the M-step's sigma^2 and c, ``em_mstep_sums``),
  the per-patch potentials p-bar for the patch mixture (an all-gather of one
  float per patch), and one sum over ranks of the adjoint volumes addon and
  conf before the SIRT update (``allreduce_sum_``).

All functions here are plain host code over numpy arrays or torch tensors and
any torch.distributed process group.
"""
from __future__ import annotations

import numpy as np

DESC_COLS = 8       # stack, slice, x0, y0, w, h, pix_off, reserved


def partition_by_pixels(desc: np.ndarray, world_size: int) -> np.ndarray:
    """Row bounds [world_size + 1] of contiguous patch ranges with balanced
    pixel counts: rank r owns rows bounds[r]:bounds[r+1].

    The cut for rank r is the first row whose pixel-count prefix reaches
    r * N / world_size (integer arithmetic, so every rank computes the same
    bounds).  Ranks may own zero rows when there are fewer patches than
    ranks."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    desc = np.asarray(desc)
    n = desc.shape[0]
    npix = desc[:, 4].astype(np.int64) * desc[:, 5].astype(np.int64)
    prefix = np.concatenate([[0], np.cumsum(npix)])           # pixels before row i
    total = int(prefix[-1])
    bounds = np.empty(world_size + 1, dtype=np.int64)
    bounds[0], bounds[-1] = 0, n
    for r in range(1, world_size):
        target = (total * r) // world_size
        bounds[r] = int(np.searchsorted(prefix[:n], target, side="left"))
    return np.maximum.accumulate(bounds)


def shard_table(desc: np.ndarray, bounds: np.ndarray, rank: int):
    """Rows of `rank` with pixel offsets rebased to 0, plus the pixel range
    [lo, hi) those rows occupy in the unsharded pixel arrays.

    Requires the unsharded table to be packed (row i's pixels start where
    row i-1's end), as every patch-table builder here produces."""
    a, b = int(bounds[rank]), int(bounds[rank + 1])
    d = np.array(desc[a:b], dtype=np.int32, copy=True)
    if d.shape[0] == 0:
        return d.reshape(0, DESC_COLS), 0, 0
    lo = int(d[0, 6])
    npix = d[:, 4].astype(np.int64) * d[:, 5].astype(np.int64)
    if not np.array_equal(d[:, 6].astype(np.int64) - lo, np.concatenate([[0], np.cumsum(npix)[:-1]])):
        raise ValueError("patch table is not packed")
    d[:, 6] -= lo
    return d, lo, lo + int(npix.sum())


def allreduce_sum_(tensors, dist, group=None):
    """In-place sum over ranks of each tensor (the adjoint volumes addon and
    conf, the EM sums).  One collective per tensor, issued in order."""
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors


def em_global_stats(e, valid, dist, group=None):
    """Global statistics of the residuals for the EM initialisation and the
    uniform outlier density m = 1 / (max e - min e): returns
    (n_valid, sum e^2, e_min, e_max) over the valid pixels of all ranks, as
    float64 (counts are exact below 2^53)."""
    import torch
    e = torch.as_tensor(e, dtype=torch.float64)
    v = torch.as_tensor(valid).to(torch.bool)
    ev = e[v]
    s = torch.tensor([float(ev.numel()), float((ev * ev).sum())], dtype=torch.float64)
    big = torch.finfo(torch.float64).max
    lo = torch.tensor([float(ev.min()) if ev.numel() else big], dtype=torch.float64)
    hi = torch.tensor([float(ev.max()) if ev.numel() else -big], dtype=torch.float64)
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(lo, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(hi, op=dist.ReduceOp.MAX, group=group)
    return float(s[0]), float(s[1]), float(lo[0]), float(hi[0])


def em_mstep_sums(p, e, valid, dist, group=None):
    """Global M-step sums after the E-step (Sec. II, EM outlier model: the
    new sigma^2 = sum p e^2 / sum p and c = sum p / N): returns (sum p,
    sum p e^2) over the valid participating pixels of all ranks, float64."""
    import torch
    p = torch.as_tensor(p, dtype=torch.float64)
    e = torch.as_tensor(e, dtype=torch.float64)
    v = torch.as_tensor(valid).to(torch.bool)
    s = torch.tensor([float(p[v].sum()), float((p[v] * e[v] * e[v]).sum())], dtype=torch.float64)
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    return float(s[0]), float(s[1])


def gather_patch_values(vals, bounds, dist, group=None):
    """All-gather a per-patch vector (e.g. p-bar) from the ranks' row ranges
    into the unsharded order.  Ranks own unequal row counts, so every rank
    pads to the longest range."""
    import torch
    ws = len(bounds) - 1
    counts = np.diff(bounds)
    m = int(max(counts.max(), 1))
    v = torch.as_tensor(vals, dtype=torch.float64).reshape(-1)
    pad = torch.zeros(m, dtype=torch.float64)
    pad[:v.numel()] = v
    out = [torch.zeros(m, dtype=torch.float64) for _ in range(ws)]
    dist.all_gather(out, pad, group=group)
    return torch.cat([out[r][:int(counts[r])] for r in range(ws)]).numpy()


def max_over_ranks(value: float, dist, device="cpu", group=None) -> float:
    """The slowest rank's time: the job's wall time for one timed region."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
