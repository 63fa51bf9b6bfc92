"""Pins of the oracle's EM weights, SIRT update, NCC/registration and metrics
against facts fixed by statistics and algebra (not by re-typing formulas):

* EM on residuals drawn from a known Gaussian + uniform mixture recovers
  sigma and the inlier proportion c within sampling error;
* degenerate cases: constant residuals -> m = 0 -> p = 1; p lies in [0, 1] and
  decreases with |e|;
* patch potentials: all-inlier patches have p-bar = 1 exactly when m = 0;
  planted outlier patches (a heavy-tailed residual population) are masked;
* SIRT on a consistent system (y = A x*) reduces the data residual
  monotonically and keeps x >= 0;
* the edge-preserving diffusion step after it: the identity for lambda = 0,
  a constant and a linear ramp are fixed points, total intensity is
  conserved, for a large edge threshold it is the linear 26-neighbour
  diffusion (scipy correlate with the same weights), and a large step edge
  is smoothed far less than a small one;
* NCC: self-similarity 1, invariance to positive affine intensity changes,
  sign flip for negative scaling; gradient = central finite differences;
* noiseless registration recovers a known rigid transform, and a known
  affine one (12 parameters; the affine gradient equals central finite
  differences too);
* PSNR of a known MSE, CC/SSIM of identical images.
"""
import math

import numpy as np
import pytest

from oracle import pvr_oracle as O
from paper_1611_07289_b300 import synth


def _one_patch_desc(P, n):
    return np.array([[0, 0, 0, 0, n, 1, p * n, 0] for p in range(P)], dtype=np.int32)


def test_em_recovers_mixture_parameters():
    rng = np.random.default_rng(0)
    n = 200_000
    sigma_t, c_t, lo, hi = 7.0, 0.8, -400.0, 400.0
    inl = rng.uniform(size=n) < c_t
    e = np.where(inl, rng.normal(0, sigma_t, n), rng.uniform(lo, hi, n))
    e[0], e[1] = lo, hi  # pin the range so m = 1 / (hi - lo)
    desc = _one_patch_desc(1, n)
    y = e.astype(np.float32)
    sim = np.zeros(n)
    valid = np.ones(n, dtype=np.uint8)
    st = O.new_state()
    ep = O.em_params(c0=0.5)
    for _ in range(60):
        O.em_weights(y, sim, valid, desc, ep, st)
    sigma = math.sqrt(st[O.ST["SIGMA2"]])
    c = st[O.ST["C"]]
    assert abs(st[O.ST["M"]] - 1.0 / (hi - lo)) < 1e-12
    assert abs(sigma - sigma_t) < 0.05 * sigma_t
    assert abs(c - c_t) < 0.01


def test_em_degenerate_and_monotone():
    n = 64
    desc = _one_patch_desc(1, n)
    valid = np.ones(n, dtype=np.uint8)
    st = O.new_state()
    p, wp, pbar, mask = O.em_weights(np.full(n, 3.0, np.float32), np.zeros(n), valid, desc,
                                     O.em_params(), st)
    assert st[O.ST["M"]] == 0.0 and np.all(p == 1.0) and pbar[0] == 1.0
    e = np.linspace(-50, 50, n)
    st = O.new_state()
    p, _, _, _ = O.em_weights(e.astype(np.float32), np.zeros(n), valid, desc, O.em_params(), st)
    assert np.all((p >= 0) & (p <= 1))
    a = np.abs(e)
    order = np.argsort(a)
    assert np.all(np.diff(p[order]) <= 1e-15)
    # invalid pixels get p = 0 and do not enter the statistics
    valid2 = valid.copy()
    valid2[:8] = 0
    st2 = O.new_state()
    p2, _, _, _ = O.em_weights(e.astype(np.float32), np.zeros(n), valid2, desc, O.em_params(), st2)
    assert np.all(p2[:8] == 0) and st2[O.ST["N_PART"]] == n - 8


def test_planted_outlier_patches_are_masked():
    rng = np.random.default_rng(1)
    P, n = 60, 400
    bad = set(rng.choice(P, 6, replace=False).tolist())
    e = np.empty(P * n)
    for s in range(P):
        if s in bad:
            e[s * n:(s + 1) * n] = rng.normal(0, 150.0, n)   # misregistered / corrupted
        else:
            e[s * n:(s + 1) * n] = rng.normal(0, 10.0, n)
    desc = _one_patch_desc(P, n)
    st = O.new_state()
    mask = None
    for _ in range(5):
        p, wp, pbar, mask = O.em_weights(e.astype(np.float32), np.zeros(P * n),
                                         np.ones(P * n, np.uint8), desc, O.em_params(), st, mask)
    got_bad = {s for s in range(P) if mask[s] == 0}
    assert got_bad == bad
    assert all(pbar[s] < min(pbar[t] for t in range(P) if t not in bad) for s in bad)
    # threshold rule: same classification with a threshold between the groups
    thr = 0.5 * (max(pbar[s] for s in bad) + min(pbar[t] for t in range(P) if t not in bad))
    st1 = O.new_state()
    _, w1, pb1, m1 = O.em_weights(e.astype(np.float32), np.zeros(P * n), np.ones(P * n, np.uint8),
                                  desc, O.em_params(patch_rule=1, patch_threshold=thr), st1, mask)
    assert {s for s in range(P) if m1[s] == 0} == bad


def test_patch_with_few_valid_pixels_is_excluded():
    P, n = 4, 100
    desc = _one_patch_desc(P, n)
    valid = np.ones(P * n, np.uint8)
    valid[0:95] = 0  # patch 0: 5 % valid (< 10 %)
    rng = np.random.default_rng(2)
    e = rng.normal(0, 5, P * n).astype(np.float32)
    st = O.new_state()
    _, wp, _, mask = O.em_weights(e, np.zeros(P * n), valid, desc, O.em_params(), st)
    assert mask[0] == 0 and wp[0] == 0.0 and st[O.ST["N_ELIG"]] == 3


def test_sirt_reduces_residual_on_consistent_data():
    rng = np.random.default_rng(7)
    geom = synth.random_geometry(rng, n=12, n_stacks=3, W=10, H=10, K=6, thick=2.0)
    desc, npix = synth.all_patches(geom, 5, 5)
    poses = synth.random_poses(rng, desc.shape[0], rot=3.0, trans=0.5)
    G = O.geom(geom)
    ps = O.psf(1.2, 1, 2, 1.0)
    fix = O.pose_fixed(G, ps, desc, poses)
    xt = rng.uniform(0, 100, geom.n_vox).astype(np.float32)
    y, valid, _ = O.simulate(G, ps, xt, desc, fix, npix)
    x = O.volume_init(G, ps, desc, fix, y)
    prev = None
    for _ in range(8):
        s, _, _ = O.simulate(G, ps, x.astype(np.float32), desc, fix, npix)
        res = np.linalg.norm((y - s)[valid > 0])
        if prev is not None:
            assert res < prev
        prev = res
        addon, conf = O.adjoint(G, ps, desc, fix, r=np.where(valid > 0, y - s, 0.0), w=None)
        x = O.volume_update(x, addon, conf, 1.0)
        assert np.all(x >= 0)


def test_sirt_step_maps_constant_data_to_the_constant():
    """Rows of A sum to one, so for y = c on every valid pixel one SIRT step
    from x = 0 gives x = c exactly on every voxel a sample reached."""
    rng = np.random.default_rng(8)
    geom = synth.random_geometry(rng, n=10, n_stacks=3, W=8, H=8, K=4, thick=2.0)
    desc, npix = synth.all_patches(geom, 4, 2)
    poses = synth.random_poses(rng, desc.shape[0], rot=10.0, trans=1.0)
    G = O.geom(geom)
    ps = O.psf(1.2, 1, 2, 1.0)
    fix = O.pose_fixed(G, ps, desc, poses)
    _, valid, _ = O.simulate(G, ps, np.zeros(geom.n_vox, np.float32), desc, fix, npix)
    r = np.where(valid > 0, 250.0, 0.0)
    w = rng.uniform(0.2, 1.0, npix)
    addon, conf = O.adjoint(G, ps, desc, fix, r=r, w=w)
    x1 = O.volume_update(np.zeros(geom.n_vox), addon, conf, 1.0, 1e-6)
    reached = conf > 1e-6
    assert reached.sum() > 100
    np.testing.assert_allclose(x1[reached], 250.0, rtol=1e-12)
    assert np.all(x1[~reached] == 0.0)


def _reg_case(seed=0):
    cfg = synth.config_tiny(seed=1611, noise=False)
    geom = cfg["geom"]
    x = cfg["gt"].reshape(-1)
    rng = np.random.default_rng(seed)
    desc, npix = synth.all_patches(geom, 32, 16)
    # central patches: their PSF samples stay inside the volume for the poses
    # used here, where NCC is a smooth function of the pose (a sample leaving
    # the volume changes the normalisation discontinuously)
    central = np.flatnonzero((desc[:, 2] == 16) & (desc[:, 3] == 16) & (desc[:, 1] >= 5)
                             & (desc[:, 1] <= 14))
    sel = rng.choice(central, 6, replace=False)
    d = desc[sel].copy()
    off = 0
    for r in d:
        r[6] = off
        off += int(r[4] * r[5])
    return geom, x, d, off


def _sr(u, lam, delta, conf=None, addon=None):
    nz, ny, nx = u.shape
    conf = np.ones(u.size) if conf is None else conf
    addon = np.zeros(u.size) if addon is None else addon
    return O.sr_update(u.reshape(-1), addon, conf, (nx, ny, nz), 1.0, 1e-6, lam, delta).reshape(u.shape)


def test_sr_update_fixed_points_and_identity():
    rng = np.random.default_rng(0)
    u = rng.uniform(100, 900, (6, 7, 8))
    addon = rng.normal(0, 30, u.size)
    conf = rng.uniform(0.0, 2.0, u.size)
    conf[::7] = 0.0
    # lambda = 0: exactly the SIRT step
    assert np.array_equal(O.sr_update(u.reshape(-1), addon, conf, (8, 7, 6), 1.0, 1e-6, 0.0, 50.0),
                          O.volume_update(u.reshape(-1), addon, conf))
    # a constant volume is a fixed point
    c = np.full((6, 7, 8), 321.0)
    assert np.array_equal(_sr(c, 0.8, 20.0), c)
    # a linear ramp is a fixed point away from the border (fluxes of opposite
    # neighbours cancel), for any edge threshold
    z, y, x = np.meshgrid(np.arange(6), np.arange(7), np.arange(8), indexing="ij")
    ramp = 200.0 + 13.0 * x - 7.0 * y + 5.0 * z
    for delta in (3.0, 1e6):
        out = _sr(ramp, 0.7, delta)
        assert np.allclose(out[1:-1, 1:-1, 1:-1], ramp[1:-1, 1:-1, 1:-1], rtol=0, atol=1e-10)
        assert not np.allclose(out, ramp, rtol=0, atol=1e-6)   # the border does move


def test_sr_update_conserves_intensity_and_is_linear_diffusion_for_large_delta():
    from scipy.ndimage import correlate
    rng = np.random.default_rng(1)
    u = rng.uniform(400, 600, (9, 10, 11))
    out = _sr(u, 0.5, 25.0)
    assert abs(out.sum() - u.sum()) <= 1e-12 * u.sum()
    # edge threshold far above every difference: psi(D) = D exactly, the
    # step is (1 - lambda) u + lambda * (26-neighbour weighted mean)
    k = np.zeros((3, 3, 3))
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                r2 = dx * dx + dy * dy + dz * dz
                if r2:
                    k[dz + 1, dy + 1, dx + 1] = (1.0 / r2) / (6 + 12 / 2 + 8 / 3)
    lam = 0.6
    lin = _sr(u, lam, 1e30)
    ref = (1 - lam) * u + lam * correlate(u, k, mode="constant")
    assert np.allclose(lin[1:-1, 1:-1, 1:-1], ref[1:-1, 1:-1, 1:-1], rtol=1e-13, atol=0)


def test_sr_update_preserves_large_edges():
    """Edge-stopping flux: a step of 10 delta moves by a few per cent of what
    a step of delta / 10 moves, relative to its height."""
    def edge_change(h):
        u = np.full((4, 6, 8), 500.0)
        u[:, :, 4:] += h
        out = _sr(u, 0.8, 10.0)
        return np.max(np.abs(out - u)) / h
    small, large = edge_change(1.0), edge_change(100.0)
    assert large < 0.15 * small, (small, large)


def test_ncc_identities():
    geom, x, d, npix = _reg_case()
    G = O.geom(geom)
    ps = O.psf(1.2, 1, 3, 1.0)
    th = np.zeros((d.shape[0], 6))
    th[:, 3:] = 2.0
    fix = O.pose_fixed(G, ps, d, th)
    y, valid, _ = O.simulate(G, ps, x, d, fix, npix)
    for s in range(d.shape[0]):
        off = int(d[s, 6])
        ys = y[off:off + 1024]
        for scale, shift, expect in ((1.0, 0.0, 1.0), (2.5, 40.0, 1.0), (-1.0, 500.0, -1.0)):
            yy = np.zeros(npix, np.float32)
            yy[off:off + 1024] = (scale * ys + shift).astype(np.float32)
            v, _ = O.ncc_grad(G, ps, x, yy, d[s], th[s])
            assert abs(v - expect) < 1e-6, (s, scale, v)


def test_ncc_gradient_matches_finite_differences():
    geom, x, d, npix = _reg_case(1)
    G = O.geom(geom)
    ps = O.psf(1.2, 1, 3, 1.0)
    th_true = np.zeros((d.shape[0], 6))
    fix = O.pose_fixed(G, ps, d, th_true)
    y, _, _ = O.simulate(G, ps, x, d, fix, npix)
    y = y.astype(np.float32)
    rng = np.random.default_rng(3)
    h = 1e-4
    for s in range(3):
        th = th_true[s] + np.concatenate([rng.uniform(-2, 2, 3), rng.uniform(-3, 3, 3)])
        _, g = O.ncc_grad(G, ps, x, y, d[s], th, exact=False)
        fd = np.zeros(6)
        for k in range(6):
            tp, tm = th.copy(), th.copy()
            tp[k] += h
            tm[k] -= h
            fd[k] = (O.ncc_grad(G, ps, x, y, d[s], tp, exact=False)[0]
                     - O.ncc_grad(G, ps, x, y, d[s], tm, exact=False)[0]) / (2 * h)
        assert np.linalg.norm(g - fd) <= 2e-3 * np.linalg.norm(fd) + 1e-9, (g, fd)
        # the fixed-point (exact) gradient is the same quantity up to 2^-20 voxel
        _, ge = O.ncc_grad(G, ps, x, y, d[s], th, exact=True)
        assert np.linalg.norm(ge - g) <= 1e-3 * np.linalg.norm(g)


def test_noiseless_registration_recovers_known_transform():
    from scipy.ndimage import gaussian_filter
    geom, _, d, npix = _reg_case(2)
    # a textured volume makes every pose direction observable from a patch
    tex = gaussian_filter(np.random.default_rng(8).normal(size=(64, 64, 64)), 2.5)
    x = (500 + 400 * tex / tex.std()).astype(np.float32).reshape(-1)
    G = O.geom(geom)
    ps = O.psf(1.2, 1, 3, 1.0)
    rng = np.random.default_rng(4)
    th_true = np.concatenate([rng.uniform(-1, 1, (d.shape[0], 3)), rng.uniform(-2, 2, (d.shape[0], 3))], 1)
    fix = O.pose_fixed(G, ps, d, th_true)
    y, _, _ = O.simulate(G, ps, x, d, fix, npix)
    start = th_true + np.concatenate([rng.uniform(-3, 3, (d.shape[0], 3)),
                                      rng.uniform(-5, 5, (d.shape[0], 3))], 1)
    rp = O.reg_params(n_eval=200, delta0=2.0, delta_min=1e-4)
    got, ncc = O.register(G, ps, rp, x, y.astype(np.float32), d, start)
    err_t = np.abs(got[:, :3] - th_true[:, :3]).max()
    err_r = np.abs(got[:, 3:] - th_true[:, 3:]).max()
    assert np.all(ncc > 0.999)
    assert err_t < 0.1 and err_r < 0.1, (err_t, err_r)


def test_affine_ncc_gradient_matches_finite_differences():
    geom, x, d, npix = _reg_case(1)
    G = O.geom(geom)
    ps = O.psf(1.2, 1, 3, 1.0)
    fix = O.pose_fixed(G, ps, d, np.zeros((d.shape[0], 6)))
    y, _, _ = O.simulate(G, ps, x, d, fix, npix)
    y = y.astype(np.float32)
    rng = np.random.default_rng(13)
    h = 1e-5
    for s in range(3):
        th = np.concatenate([rng.uniform(-2, 2, 3), rng.uniform(-0.05, 0.05, 9)])
        _, g = O.ncc_grad(G, ps, x, y, d[s], th, n_params=12, exact=False)
        fd = np.zeros(12)
        for k in range(12):
            tp, tm = th.copy(), th.copy()
            tp[k] += h
            tm[k] -= h
            fd[k] = (O.ncc_grad(G, ps, x, y, d[s], tp, n_params=12, exact=False)[0]
                     - O.ncc_grad(G, ps, x, y, d[s], tm, n_params=12, exact=False)[0]) / (2 * h)
        assert np.linalg.norm(g - fd) <= 2e-3 * np.linalg.norm(fd) + 1e-9, (g, fd)
        # the D entries move samples by (w - c), so their gradient is far from zero
        assert np.linalg.norm(g[3:]) > 10 * np.linalg.norm(g[:3]) * 1e-3


def test_noiseless_affine_registration_recovers_known_transform():
    from scipy.ndimage import gaussian_filter
    geom, _, d, npix = _reg_case(2)
    tex = gaussian_filter(np.random.default_rng(8).normal(size=(64, 64, 64)), 2.5)
    x = (500 + 400 * tex / tex.std()).astype(np.float32).reshape(-1)
    G = O.geom(geom)
    ps = O.psf(1.2, 1, 3, 1.0)
    rng = np.random.default_rng(14)
    P = d.shape[0]
    # a stretch / shear of a few per cent (breathing-like), the in-plane part
    # observable from a 2-D patch; the out-of-plane column of D moves
    # samples only by zeta steps (weakly observable) and stays at its truth
    th_true = np.concatenate([rng.uniform(-1, 1, (P, 3)), rng.uniform(-0.04, 0.04, (P, 9))], 1)
    fix = O.pose_fixed(G, ps, d, th_true, n_params=12)
    y, _, _ = O.simulate(G, ps, x, d, fix, npix)
    start = th_true.copy()
    start[:, :3] += rng.uniform(-2, 2, (P, 3))
    start[:, 3:] += rng.uniform(-0.04, 0.04, (P, 9))
    rp = O.reg_params(n_params=12, n_eval=400, delta0=2.0, delta_min=1e-5)
    got, ncc = O.register(G, ps, rp, x, y.astype(np.float32), d, start)
    assert np.all(ncc > 0.9999)
    # residual displacement over the patch: |dt + dD (w - c)| at the patch corners (mm)
    for s in range(P):
        S = np.asarray(geom.p2w[int(d[s, 0])])
        half = np.array([(d[s, 4] - 1) / 2.0, (d[s, 5] - 1) / 2.0])
        dD = (got[s, 3:] - th_true[s, 3:]).reshape(3, 3)
        for sx in (-1, 1):
            for sy in (-1, 1):
                u = S[:, 0] * sx * half[0] + S[:, 1] * sy * half[1]
                disp = (got[s, :3] - th_true[s, :3]) + dD @ u
                assert np.linalg.norm(disp) < 0.05, (s, disp)


def test_metrics_closed_forms():
    rng = np.random.default_rng(0)
    ref = rng.uniform(0, 1000, 5000)
    ref[0] = 1000.0
    m = O.metrics(ref, ref + 10.0)
    assert abs(m["mse"] - 100.0) < 1e-9
    assert abs(m["psnr"] - 40.0) < 1e-9
    assert abs(m["cc"] - 1.0) < 1e-12
    s = O.metrics(ref, ref)
    assert abs(s["ssim"] - 1.0) < 1e-12 and abs(s["dssim"]) < 1e-12 and s["cc"] > 1 - 1e-12
    neg = O.metrics(ref, 2000.0 - ref)
    assert abs(neg["cc"] + 1.0) < 1e-12
    # SSIM drops below 1 for a noisy copy and DSSIM = (1 - SSIM) / 2
    n = O.metrics(ref, ref + rng.normal(0, 100, ref.size))
    assert 0 < n["ssim"] < 1 and abs(n["dssim"] - (1 - n["ssim"]) / 2) < 1e-15


def test_patch_metrics_and_local_ssim_map():
    """Identical patches: SSIM 1 everywhere, DSSIM 0.  Local SSIM of interior
    pixels equals the box-window formula built from scipy's uniform_filter
    (an independent construction of the window sums)."""
    from scipy.ndimage import uniform_filter
    rng = np.random.default_rng(21)
    desc = np.array([[0, 0, 0, 0, 20, 16, 0, 0], [0, 1, 0, 0, 9, 7, 320, 0]], dtype=np.int32)
    npix = 320 + 63
    y = rng.uniform(100, 900, npix).astype(np.float32)
    valid = np.ones(npix, np.uint8)
    out, m = O.patch_metrics(y, y, valid, desc, 3)
    assert np.allclose(out[:, 2], 1.0) and np.allclose(out[:, 4], 1.0) and np.all(m == 0.0)
    s = (y + rng.normal(0, 40, npix)).astype(np.float32)
    out, m = O.patch_metrics(y, s, valid, desc, 3)
    ref_g = O.metrics(y[:320], s[:320])
    assert abs(out[0, 0] - ref_g["psnr"]) < 1e-9 and abs(out[0, 2] - ref_g["ssim"]) < 1e-12
    a = y[:320].reshape(16, 20).astype(np.float64)
    b = s[:320].reshape(16, 20).astype(np.float64)
    f = lambda v: uniform_filter(v, size=7, mode="constant")
    ma, mb = f(a), f(b)
    va, vb, cab = f(a * a) - ma * ma, f(b * b) - mb * mb, f(a * b) - ma * mb
    L = a.max() - a.min()
    c1, c2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    ss = ((2 * ma * mb + c1) * (2 * cab + c2)) / ((ma * ma + mb * mb + c1) * (va + vb + c2))
    inner = (slice(3, 13), slice(3, 17))
    assert np.allclose(m[:320].reshape(16, 20)[inner], (1 - ss[inner]) / 2, rtol=1e-9, atol=1e-12)


def test_outer_iterations_raise_psnr_on_the_tiny_workload():
    """The whole oracle iteration (registration, EM, SIRT) improves the volume:
    on the noise-free 64^3 workload (slices moved by up to 5 degrees and 3 mm)
    PSNR against the phantom rises over the first two outer iterations (after
    that, SIRT without a regulariser semi-converges)."""
    from paper_1611_07289_b300 import synth
    cfg = synth.config_tiny(noise=False)
    geom = cfg["geom"]
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 1.0)
    desc, npix = O.patches_build(G, synth.pack_stacks(cfg["stacks"]), 32, 16)
    y = synth.pack_patch_pixels(cfg["stacks"], desc)
    poses = np.zeros((desc.shape[0], 6))
    x = O.volume_init(G, ps, desc, O.pose_fixed(G, ps, desc, poses), y).astype(np.float32)
    gt = np.asarray(cfg["gt"], np.float64).reshape(-1)

    def psnr(a):
        return 10.0 * np.log10(gt.max() ** 2 / np.mean((np.asarray(a, np.float64).reshape(-1) - gt) ** 2))

    st, mask = O.new_state(), np.ones(desc.shape[0], np.uint8)
    trace = [psnr(x)]
    for _ in range(2):
        x, poses, mask, _ = O.reconstruct_iter(G, ps, O.em_params(), O.reg_params(n_eval=10), x, y, desc, poses,
                                               npix, st, mask, n_sr=2)
        trace.append(psnr(x))
    assert trace[1] > trace[0] + 0.3 and trace[2] > trace[1], trace
