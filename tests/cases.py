"""Seeded cases shared by the GPU parity tests (inputs only; no method
arithmetic)."""
import numpy as np

from paper_1611_07289_b300 import synth


def uneven_case(seed=0, n=16, stacks=3, W=40, H=36, K=5, thick=2.0):
    """Random stacks through an n^3 volume with uneven patches (sizes 1..33,
    odd offsets), random poses."""
    rng = np.random.default_rng(seed)
    geom = synth.random_geometry(rng, n=n, n_stacks=stacks, W=W, H=H, K=K, thick=thick, pix=0.6)
    rows, off = [], 0
    for s in range(stacks):
        for k in range(K):
            for _ in range(3):
                w = int(rng.integers(1, 34))
                h = int(rng.integers(1, 34))
                x0 = int(rng.integers(0, W - w + 1))
                y0 = int(rng.integers(0, H - h + 1))
                rows.append([s, k, x0, y0, w, h, off, 0])
                off += w * h
    desc = np.array(rows, dtype=np.int32)
    poses = synth.random_poses(rng, len(rows), rot=20.0, trans=2.0)
    return geom, desc, off, poses, rng


def tiled_case(seed=1):
    """Large patches (up to 130 px) that span several 64x64 tiles with
    ragged edges."""
    rng = np.random.default_rng(seed)
    n = 24
    w2v, v2w = synth.volume_geometry((n, n, n), 1.0)
    p2w = [synth.stack_matrix(*synth.rot_zyx(*rng.uniform(-30, 30, 3)).T, 150, 140, 3, 0.15, 2.0)
           for _ in range(2)]
    geom = synth.Geometry((n, n, n), w2v, v2w, [(150, 140, 3)] * 2, p2w, [2.0, 2.0])
    sizes = [(130, 70), (100, 77), (65, 64), (64, 65), (129, 129), (3, 100)]
    rows, off = [], 0
    for i, (w, h) in enumerate(sizes):
        s, k = i % 2, i % 3
        x0 = int(rng.integers(0, 150 - w + 1))
        y0 = int(rng.integers(0, 140 - h + 1))
        rows.append([s, k, x0, y0, w, h, off, 0])
        off += w * h
    desc = np.array(rows, dtype=np.int32)
    poses = synth.random_poses(rng, len(rows), rot=10.0, trans=1.0)
    return geom, desc, off, poses, rng


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
