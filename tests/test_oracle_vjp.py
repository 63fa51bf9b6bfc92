"""Pins of the oracle's pose vector-Jacobian product of the forward model
(Eq. 1 differentiated through the sample positions), the backward pass of a
differentiable simulate:

* it equals central finite differences of its own value with FP64 sample
  positions (smooth in the pose), for rigid and affine poses;
* its value in fixed-point mode is sum r * sim of the pinned forward model;
* on a volume that is linear in the voxel coordinates trilinear
  interpolation is exact, every pixel of an in-volume patch moves by the
  same amount per millimetre of translation, and the translation gradient
  is the closed form sum_valid r * (a . column of world_to_voxel).
"""
import numpy as np

from oracle import pvr_oracle as O
from paper_1611_07289_b300 import synth


def _case(seed):
    cfg = synth.config_tiny(seed=1611, noise=False)
    geom = cfg["geom"]
    x = cfg["gt"].reshape(-1).astype(np.float32)
    desc, npix = synth.all_patches(geom, 32, 16)
    central = np.flatnonzero((desc[:, 2] == 16) & (desc[:, 3] == 16) & (desc[:, 1] >= 5)
                             & (desc[:, 1] <= 14))
    rng = np.random.default_rng(seed)
    d = desc[rng.choice(central, 4, replace=False)].copy()
    off = 0
    for r in d:
        r[6] = off
        off += int(r[4] * r[5])
    return geom, x, d, off, rng


def test_pose_vjp_matches_finite_differences():
    geom, x, d, npix, rng = _case(4)
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 1.0)
    r = rng.normal(size=npix)
    h = 1e-4
    for s in range(d.shape[0]):
        th = np.concatenate([rng.uniform(-2, 2, 3), rng.uniform(-3, 3, 3)])
        _, g = O.sim_pose_vjp(G, ps, x, r, d[s], th, exact=False)
        fd = np.zeros(6)
        for k in range(6):
            tp, tm = th.copy(), th.copy()
            tp[k] += h
            tm[k] -= h
            fd[k] = (O.sim_pose_vjp(G, ps, x, r, d[s], tp, exact=False)[0]
                     - O.sim_pose_vjp(G, ps, x, r, d[s], tm, exact=False)[0]) / (2 * h)
        assert np.linalg.norm(g - fd) <= 2e-3 * np.linalg.norm(fd) + 1e-9, (g, fd)
        _, ge = O.sim_pose_vjp(G, ps, x, r, d[s], th, exact=True)
        assert np.linalg.norm(ge - g) <= 1e-3 * np.linalg.norm(g)


def test_affine_pose_vjp_matches_finite_differences():
    geom, x, d, npix, rng = _case(6)
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 1.0)
    r = rng.normal(size=npix)
    h = 1e-5
    for s in range(2):
        th = np.concatenate([rng.uniform(-2, 2, 3), rng.uniform(-0.05, 0.05, 9)])
        _, g = O.sim_pose_vjp(G, ps, x, r, d[s], th, n_params=12, exact=False)
        fd = np.zeros(12)
        for k in range(12):
            tp, tm = th.copy(), th.copy()
            tp[k] += h
            tm[k] -= h
            fd[k] = (O.sim_pose_vjp(G, ps, x, r, d[s], tp, n_params=12, exact=False)[0]
                     - O.sim_pose_vjp(G, ps, x, r, d[s], tm, n_params=12, exact=False)[0]) / (2 * h)
        assert np.linalg.norm(g - fd) <= 2e-3 * np.linalg.norm(fd) + 1e-9, (g, fd)


def test_pose_vjp_value_is_the_forward_model():
    geom, x, d, npix, rng = _case(5)
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 1.0)
    poses = synth.random_poses(rng, d.shape[0], rot=4.0, trans=2.0)
    fix = O.pose_fixed(G, ps, d, poses)
    sim, valid, _ = O.simulate(G, ps, x, d, fix, npix)
    r = rng.normal(size=npix)
    for s in range(d.shape[0]):
        o, n = int(d[s, 6]), int(d[s, 4] * d[s, 5])
        v, _ = O.sim_pose_vjp(G, ps, x, r, d[s], poses[s], exact=True)
        ref = float(np.sum(r[o:o + n] * sim[o:o + n] * valid[o:o + n]))
        assert abs(v - ref) <= 1e-12 * np.sum(np.abs(r[o:o + n] * sim[o:o + n]))


def test_translation_gradient_on_a_linear_volume_is_closed_form():
    geom, _, d, npix, rng = _case(6)
    nx, ny, nz = geom.vol_dims
    a = np.array([3.0, -2.0, 5.0])        # x(v) = a . v in voxel coordinates
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x = (a[0] * xx + a[1] * yy + a[2] * zz).astype(np.float32).reshape(-1)
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 1.0)
    W = np.asarray(geom.w2v, dtype=np.float64).reshape(-1)[:12].reshape(3, 4)
    r = rng.normal(size=npix)
    for s in range(d.shape[0]):
        th = np.concatenate([rng.uniform(-1, 1, 3), rng.uniform(-2, 2, 3)])
        fix = O.pose_fixed(G, ps, d[s:s + 1], th[None])
        drow = d[s:s + 1].copy()
        o, n = int(drow[0, 6]), int(drow[0, 4] * drow[0, 5])
        drow[0, 6] = 0
        _, valid, _ = O.simulate(G, ps, x, drow, fix, n)
        _, g = O.sim_pose_vjp(G, ps, x, r, d[s], th, exact=False)
        rv = float(np.sum(r[o:o + n] * valid))
        want = np.array([rv * float(a @ W[:, k]) for k in range(3)])
        assert np.allclose(g[:3], want, rtol=1e-9, atol=1e-9 * np.abs(want).max())
