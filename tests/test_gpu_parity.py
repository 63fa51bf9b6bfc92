"""GPU parity: every C-ABI entry point against the FP64 oracle on the same
seeded inputs.

Tolerances (FP32 kernels vs the FP64 oracle): relative L2 1e-5 for the
forward model and adjoint, 1e-4 for a full reconstruction iteration,
bit-exact for the fixed-point sample lattice, the valid masks and the patch
table; EM masks exact except where the oracle's patch weight lies within
1e-4 of the 0.5 decision (then both outcomes are valid)."""
import numpy as np
import pytest
import torch

from oracle import pvr_oracle as O
from paper_1611_07289_b300 import synth
from tests.cases import rel_l2, tiled_case, uneven_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pvr():
    from paper_1611_07289_b300 import pvr as m
    return m


def _ctx(pvr, geom, kxy=1, kz=3, dz=1.0, **kw):
    prm = pvr.default_params(psf_kxy=kxy, psf_kz=kz, psf_dz=dz, max_patches=4096,
                             max_pixels=1 << 22, max_patch_side=256, **kw)
    return pvr.Context(geom, prm)


def _t(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


CASES = {"uneven": uneven_case, "tiled": tiled_case}


@pytest.mark.parametrize("case", ["uneven", "tiled"])
def test_pose_to_fixed_is_bit_exact(pvr, case):
    geom, desc, npix, poses, rng = CASES[case]()
    special = [0.0, 90.0, -90.0, 180.0, 45.0, -45.0, 135.0, 270.0, 1e-9, 359.999999]
    poses = poses.copy()
    for i, a in enumerate(special):
        poses[i % len(poses), 3 + i % 3] = a
    big = synth.random_poses(rng, len(poses), rot=180.0, trans=5.0)
    for ps in (poses, big):
        ctx = _ctx(pvr, geom, dz=0.7)
        pt = pvr.PatchTable.from_numpy(desc, npix)
        fix = ctx.pvr_pose_to_fixed(pt, _t(ps)).cpu().numpy()
        ref = O.pose_fixed(O.geom(geom), O.psf(1.2, 1, 3, 0.7), desc, ps)
        assert np.array_equal(fix[:, :13].astype(np.int64), ref[:, :13])
        assert np.all(fix[:, 13] == 1)
        ctx.pvr_device_status()


@pytest.mark.parametrize("case,kxy,kz", [("uneven", 1, 3), ("uneven", 0, 0), ("uneven", 2, 5),
                                         ("tiled", 1, 3), ("tiled", 1, 1)])
def test_simulate_matches_oracle(pvr, case, kxy, kz):
    geom, desc, npix, poses, rng = CASES[case]()
    x = rng.uniform(0, 1000, geom.n_vox).astype(np.float32)
    ctx = _ctx(pvr, geom, kxy, kz, 0.8)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    sim, valid = ctx.pvr_simulate(_t(x), pt, _t(poses))
    G, ps = O.geom(geom), O.psf(1.2, kxy, kz, 0.8)
    fix = O.pose_fixed(G, ps, desc, poses)
    rs, rv, _ = O.simulate(G, ps, x, desc, fix, npix)
    sim, valid = sim.cpu().numpy(), valid.cpu().numpy()
    assert np.array_equal(valid, rv)
    assert 0.2 * npix < valid.sum() < npix
    assert rel_l2(sim, rs) < 1e-5
    ctx.pvr_device_status()


@pytest.mark.parametrize("case", ["uneven", "tiled"])
def test_taylor_sinc_psf_matches_oracle(pvr, case):
    """In-plane sinc PSF from its Taylor series (Sec. II).  Its weights have
    both signs, so the in-volume weight sum decides validity through a sum
    that can cancel: masks must agree wherever that sum is not within
    float32 rounding of zero."""
    geom, desc, npix, poses, rng = CASES[case]()
    x = rng.uniform(0, 1000, geom.n_vox).astype(np.float32)
    ctx = pvr.Context(geom, pvr.default_params(psf_kxy=3, psf_kz=3, psf_dz=0.8, psf_fwhm_xy=2.0,
                                               psf_kind=1, max_patches=4096, max_pixels=1 << 22,
                                               max_patch_side=256))
    pt = pvr.PatchTable.from_numpy(desc, npix)
    sim, valid = ctx.pvr_simulate(_t(x), pt, _t(poses))
    G, ps = O.geom(geom), O.psf(2.0, 3, 3, 0.8, kind=1)
    fix = O.pose_fixed(G, ps, desc, poses)
    rs, rv, den = O.simulate(G, ps, x, desc, fix, npix)
    sim, valid = sim.cpu().numpy(), valid.cpu().numpy()
    # no in-volume sample: the sum is exactly zero on both sides
    sure = (den == 0.0) | (np.abs(den) > 1e-5 * np.abs(den).max())
    assert np.array_equal(valid[sure], rv[sure]) and (~sure).sum() <= npix // 1000
    # s = num / den: a weight sum that cancels amplifies the float32 rounding
    # of the weights and samples by sum|g| / |den|; compare the values where
    # that factor is below 20 (the interior and most of the border)
    well = (valid == 1) & (rv == 1) & (np.abs(den) > 0.05 * np.abs(den).max())
    assert well.sum() > 0.5 * (rv == 1).sum()
    assert rel_l2(sim[well], rs[well]) < 1e-5
    # the adjoint divides by the same weight sums: the same well-conditioned pixels
    r = rng.normal(0, 50, npix).astype(np.float32) * well
    w = well.astype(np.float32)
    a, c = ctx.pvr_adjoint(pt, _t(poses), _t(r), _t(w))
    ra, rc = O.adjoint(G, ps, desc, fix, r=r.astype(np.float64), w=w.astype(np.float64))
    assert rel_l2(a.cpu().numpy(), ra) < 1e-5 and rel_l2(c.cpu().numpy(), rc) < 1e-5


@pytest.mark.parametrize("case", ["uneven", "tiled"])
def test_adjoint_matches_oracle(pvr, case):
    geom, desc, npix, poses, rng = CASES[case]()
    r = rng.normal(0, 50, npix).astype(np.float32)
    w = rng.uniform(0, 1, npix).astype(np.float32)
    ctx = _ctx(pvr, geom, 1, 3, 0.8)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    addon, conf = ctx.pvr_adjoint(pt, _t(poses), _t(r), _t(w))
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 0.8)
    fix = O.pose_fixed(G, ps, desc, poses)
    ra, rc = O.adjoint(G, ps, desc, fix, r=r.astype(np.float64), w=w.astype(np.float64))
    assert rel_l2(addon.cpu().numpy(), ra) < 1e-5
    assert rel_l2(conf.cpu().numpy(), rc) < 1e-5
    # accumulate = 1 adds on top
    a2, c2 = ctx.pvr_adjoint(pt, _t(poses), _t(r), _t(w), addon=addon.clone(), conf=conf.clone(),
                             accumulate=True)
    assert rel_l2(a2.cpu().numpy(), 2 * ra) < 1e-5
    # r = w = NULL: A^T 1
    _, c1 = ctx.pvr_adjoint(pt, _t(poses))
    _, rc1 = O.adjoint(G, ps, desc, fix)
    assert rel_l2(c1.cpu().numpy(), rc1) < 1e-5


def test_gpu_dot_product_adjoint(pvr):
    geom, desc, npix, poses, rng = tiled_case(5)
    x = rng.normal(size=geom.n_vox).astype(np.float32)
    r = rng.normal(size=npix).astype(np.float32)
    ctx = _ctx(pvr, geom)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    ax, _ = ctx.pvr_simulate(_t(x), pt, _t(poses))
    atr, _ = ctx.pvr_adjoint(pt, _t(poses), _t(r), None)
    ax, atr = ax.cpu().double().numpy(), atr.cpu().double().numpy().reshape(-1)
    lhs, rhs = float(ax @ r.astype(np.float64)), float(x.astype(np.float64) @ atr)
    assert abs(lhs - rhs) / (np.linalg.norm(ax) * np.linalg.norm(r)) < 1e-6


def test_em_weights_match_oracle(pvr):
    geom, desc, npix, poses, rng = uneven_case(3)
    P = desc.shape[0]
    y = rng.uniform(0, 1000, npix).astype(np.float32)
    sim = (y + rng.normal(0, 10, npix)).astype(np.float32)
    bad = rng.choice(P, P // 8, replace=False)
    for b in bad:
        o, n = desc[b, 6], desc[b, 4] * desc[b, 5]
        sim[o:o + n] = y[o:o + n] + rng.normal(0, 200, n).astype(np.float32)
    valid = (rng.uniform(size=npix) > 0.05).astype(np.uint8)
    ctx = _ctx(pvr, geom)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    st_g = pvr.new_state()
    st_o = O.new_state()
    mask_g = None
    mask_o = None
    ep = O.em_params()
    for it in range(3):
        p, wp, pb, mo = ctx.pvr_em_weights(_t(y), _t(sim), _t(valid), pt, st_g,
                                           mask_in=None if mask_g is None else mask_g.clone())
        rp, rwp, rpb, rmo = O.em_weights(y, sim.astype(np.float64), valid, desc, ep, st_o, mask_o)
        sg = st_g.cpu().numpy()
        for k in ("SIGMA2", "C", "M", "MU_P", "SIGMA2_P", "C_P"):
            i = O.ST[k]
            assert abs(sg[i] - st_o[i]) <= 1e-5 * max(abs(st_o[i]), 1e-12), (it, k, sg[i], st_o[i])
        assert rel_l2(p.cpu().numpy(), rp) < 1e-5
        assert rel_l2(pb.cpu().numpy(), rpb) < 1e-5
        near = np.abs(rwp - 0.5) < 1e-4
        assert np.array_equal(mo.cpu().numpy()[~near], rmo[~near])
        assert near.sum() <= 1
        mask_g, mask_o = mo, rmo
    assert 0 < rmo.sum() < P


def test_volume_update_and_init_match_oracle(pvr):
    geom, desc, npix, poses, rng = uneven_case(4)
    ctx = _ctx(pvr, geom)
    x = rng.uniform(0, 100, geom.n_vox).astype(np.float32)
    a = rng.normal(0, 10, geom.n_vox).astype(np.float32)
    c = np.where(rng.uniform(size=geom.n_vox) < 0.2, 0.0, rng.uniform(0, 3, geom.n_vox)).astype(np.float32)
    xg, ag, cg = _t(x), _t(a), _t(c)
    ctx.pvr_volume_update(xg, ag, cg, clear=True)
    ref = O.volume_update(x, a, c, 1.0, 1e-6)
    assert rel_l2(xg.cpu().numpy(), ref) < 1e-6
    assert float(ag.abs().sum()) == 0.0 and float(cg.abs().sum()) == 0.0
    y = rng.uniform(0, 1000, npix).astype(np.float32)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    x0 = ctx.pvr_volume_init(_t(y), pt, _t(poses)).cpu().numpy().reshape(-1)
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 1.0)
    fix = O.pose_fixed(G, ps, desc, poses)
    assert rel_l2(x0, O.volume_init(G, ps, desc, fix, y)) < 1e-5


def test_ncc_and_gradient_match_oracle(pvr):
    cfg = synth.config_tiny(noise=True)
    geom = cfg["geom"]
    x = cfg["gt"].reshape(-1).astype(np.float32)
    desc, npix = synth.all_patches(geom, 32, 16)
    rng = np.random.default_rng(0)
    sel = rng.choice(desc.shape[0], 40, replace=False)
    d = desc[sel].copy()
    off = 0
    for r in d:
        r[6] = off
        off += int(r[4] * r[5])
    y = synth.pack_patch_pixels(cfg["stacks"], d)
    poses = synth.random_poses(rng, len(d), rot=3.0, trans=2.0)
    ctx = _ctx(pvr, geom)
    pt = pvr.PatchTable.from_numpy(d, off)
    ncc, grad = ctx.pvr_ncc_grad(_t(x), _t(y), pt, _t(poses))
    ncc, grad = ncc.cpu().numpy(), grad.cpu().numpy()
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 1.0)
    for s in range(len(d)):
        rn, rg = O.ncc_grad(G, ps, x, y, d[s], poses[s])
        assert abs(ncc[s] - rn) < 2e-5, (s, ncc[s], rn)
        if rn != 0.0:
            assert np.linalg.norm(grad[s] - rg) <= 2e-3 * np.linalg.norm(rg) + 1e-9, (s, grad[s], rg)


def test_register_fixed_step_matches_oracle(pvr):
    cfg = synth.config_tiny(noise=False)
    geom = cfg["geom"]
    x = cfg["gt"].reshape(-1).astype(np.float32)
    desc, npix = synth.all_patches(geom, 32, 16)
    y = synth.pack_patch_pixels(cfg["stacks"], desc)
    poses = np.zeros((desc.shape[0], 6))
    ctx = _ctx(pvr, geom, reg_fixed_step=1, reg_delta0=0.5)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    pg = _t(poses)
    _, ncc = ctx.pvr_register(_t(x), _t(y), pt, pg, 4)
    rp, rn = O.register(O.geom(geom), O.psf(1.2, 1, 3, 1.0),
                        O.reg_params(n_eval=4, fixed_step=1, delta0=0.5), x, y, desc, poses)
    # Each fixed step moves delta0 along g/|g|; a gradient error e (relative)
    # turns the direction by up to e, so after 3 steps the poses agree to
    # 3 * delta0 * e.  With the float32 gradient's e <= 1e-2 (it is a sum of
    # cancelling contributions) that bounds the difference by 1.5e-2; most
    # patches agree far better.
    d = np.abs(pg.cpu().numpy() - rp).max(1)
    assert d.max() < 1.5e-2, d.max()
    assert np.quantile(d, 0.95) < 2e-3, np.quantile(d, 0.95)
    # the NCC the GPU reports is the oracle's NCC at the GPU's own final poses
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 1.0)
    ng, pgn = ncc.cpu().numpy(), pg.cpu().numpy()
    for s in range(desc.shape[0]):
        v, _ = O.ncc_grad(G, ps, x, y, desc[s], pgn[s])
        assert abs(ng[s] - v) < 2e-5, (s, ng[s], v)
    assert np.max(np.abs(ng - rn)) < 2e-3


def test_register_recovers_known_transform(pvr):
    from scipy.ndimage import gaussian_filter
    cfg = synth.config_tiny(noise=False)
    geom = cfg["geom"]
    tex = gaussian_filter(np.random.default_rng(8).normal(size=(64, 64, 64)), 2.5)
    x = (500 + 400 * tex / tex.std()).astype(np.float32).reshape(-1)
    desc, _ = synth.all_patches(geom, 32, 16)
    central = np.flatnonzero((desc[:, 2] == 16) & (desc[:, 3] == 16) & (desc[:, 1] >= 5) & (desc[:, 1] <= 14))
    d = desc[central].copy()
    for i, r in enumerate(d):
        r[6] = i * 1024
    npix = len(d) * 1024
    rng = np.random.default_rng(4)
    th_true = np.concatenate([rng.uniform(-1, 1, (len(d), 3)), rng.uniform(-2, 2, (len(d), 3))], 1)
    ctx = _ctx(pvr, geom, reg_delta_min=1e-4)
    pt = pvr.PatchTable.from_numpy(d, npix)
    y, _ = ctx.pvr_simulate(_t(x), pt, _t(th_true))
    start = th_true + np.concatenate([rng.uniform(-3, 3, (len(d), 3)), rng.uniform(-5, 5, (len(d), 3))], 1)
    pg = _t(start)
    _, ncc = ctx.pvr_register(_t(x), y, pt, pg, 200)
    got = pg.cpu().numpy()
    assert np.all(ncc.cpu().numpy() > 0.999)
    assert np.abs(got - th_true).max() < 0.1


def test_reconstruct_iter_matches_oracle(pvr):
    cfg = synth.config_tiny()
    geom = cfg["geom"]
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 1.0)
    desc, npix = O.patches_build(G, synth.pack_stacks(cfg["stacks"]), 32, 16)
    y = synth.pack_patch_pixels(cfg["stacks"], desc)
    poses = np.zeros((desc.shape[0], 6))
    fix0 = O.pose_fixed(G, ps, desc, poses)
    x0 = O.volume_init(G, ps, desc, fix0, y).astype(np.float32)
    ctx = _ctx(pvr, geom, reg_fixed_step=1, reg_delta0=0.25, reg_evals=3, n_sr=2)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    xg, pg = _t(x0.reshape(64, 64, 64)), _t(poses)
    st = pvr.new_state()
    mask = torch.ones(desc.shape[0], dtype=torch.uint8, device="cuda")
    w_patch = torch.empty(desc.shape[0], dtype=torch.float32, device="cuda")
    ctx.pvr_reconstruct_iter(xg, _t(y), pt, pg, st, mask, None, w_patch)
    ctx.pvr_device_status()
    st_o = O.new_state()
    xo, po, mo, _ = O.reconstruct_iter(G, ps, O.em_params(),
                                       O.reg_params(n_eval=3, fixed_step=1, delta0=0.25), x0, y,
                                       desc, poses, npix, st_o, np.ones(desc.shape[0], np.uint8),
                                       n_sr=2)
    assert np.max(np.abs(pg.cpu().numpy() - po)) < 1e-3
    assert rel_l2(xg.cpu().numpy(), xo) < 1e-4
    assert np.array_equal(mask.cpu().numpy(), mo)


def test_patch_table_and_gather_are_exact(pvr):
    cfg = synth.config_tiny()
    geom = cfg["geom"]
    packed = synth.pack_stacks(cfg["stacks"])
    ctx = _ctx(pvr, geom)
    for fg, keep in ((0.0, 0.0), (0.3, 0.5), (0.5, 0.9)):
        pt, n = ctx.pvr_patches_build(_t(packed), 32, 16, fg, keep)
        ref, rn = O.patches_build(O.geom(geom), packed, 32, 16, fg, keep)
        assert n == ref.shape[0] and pt.n_pix == rn
        assert np.array_equal(pt.desc.cpu().numpy(), ref)
        if n:
            y = ctx.pvr_patches_gather(_t(packed), pt)
            assert np.array_equal(y.cpu().numpy(), synth.pack_patch_pixels(cfg["stacks"], ref))


def test_metrics_match_oracle(pvr):
    rng = np.random.default_rng(0)
    ref = rng.uniform(0, 1000, 100_003).astype(np.float32)
    img = (ref + rng.normal(0, 30, ref.size)).astype(np.float32)
    geom, *_ = uneven_case(0)
    ctx = _ctx(pvr, geom)
    out = ctx.pvr_metrics(_t(ref), _t(img)).cpu().numpy()
    m = O.metrics(ref, img)
    for i, k in enumerate(("psnr", "cc", "ssim", "dssim", "mse")):
        assert abs(out[i] - m[k]) <= 1e-9 * max(1.0, abs(m[k])), k
