"""Affine patch poses on the GPU (12 parameters: translation and the matrix
D of T(w) = (I + D)(w - c) + c + t; Eq. 1's T_i under affine motion,
Sec. II) against the FP64 oracle, whose affine path is pinned on the CPU by
an independent dense-operator construction, a numpy composition of the
lattice, finite differences and noiseless recovery.

Tolerances as for rigid poses: the fixed-point lattice and valid masks
bit-exact, forward model and adjoint relative L2 1e-5, NCC 2e-5 absolute,
pose gradients 2e-3 relative (12 components)."""
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


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _ctx(pvr, geom, dz=0.8, **kw):
    prm = pvr.default_params(psf_dz=dz, max_patches=4096, max_pixels=1 << 22, max_patch_side=256,
                             n_params=12, **kw)
    return pvr.Context(geom, prm)


def _affine(rng, n, dmax=0.1, trans=2.0):
    return np.concatenate([rng.uniform(-trans, trans, (n, 3)), rng.uniform(-dmax, dmax, (n, 9))], 1)


CASES = {"uneven": uneven_case, "tiled": tiled_case}


@pytest.mark.parametrize("case", ["uneven", "tiled"])
def test_affine_lattice_is_bit_exact(pvr, case):
    geom, desc, npix, _, rng = CASES[case]()
    poses = _affine(rng, desc.shape[0])
    poses[0, 3:] = 0.0                      # identity linear part
    poses[1, 3:] = [-0.5, 0, 0, 0, 0.25, 0, 0, 0, 2.0]   # axis scalings
    poses[2, 3:] = [0, 0.3, 0, -0.3, 0, 0, 0, 0, 0]       # skew
    ctx = _ctx(pvr, geom, dz=0.7)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    fix = ctx.pvr_pose_to_fixed(pt, _t(poses)).cpu().numpy()
    ref = O.pose_fixed(O.geom(geom), O.psf(1.2, 1, 3, 0.7), desc, poses, n_params=12)
    assert np.array_equal(fix[:, :13].astype(np.int64), ref[:, :13])
    assert np.all(fix[:, 13] == 1)
    ctx.pvr_device_status()


@pytest.mark.parametrize("case", ["uneven", "tiled"])
def test_affine_simulate_and_adjoint_match_oracle(pvr, case):
    geom, desc, npix, _, rng = CASES[case]()
    poses = _affine(rng, desc.shape[0])
    x = rng.uniform(0, 1000, geom.n_vox).astype(np.float32)
    r = rng.normal(size=npix).astype(np.float32)
    w = rng.uniform(0, 1, npix).astype(np.float32)
    ctx = _ctx(pvr, geom)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    sim, valid = ctx.pvr_simulate(_t(x), pt, _t(poses))
    addon, conf = ctx.pvr_adjoint(pt, _t(poses), _t(r), _t(w))
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 0.8)
    fix = O.pose_fixed(G, ps, desc, poses, n_params=12)
    rs, rv, _ = O.simulate(G, ps, x, desc, fix, npix)
    ra, rc = O.adjoint(G, ps, desc, fix, r=r.astype(np.float64), w=w.astype(np.float64))
    assert rv.sum() > 0.3 * npix
    assert np.array_equal(valid.cpu().numpy(), rv)
    assert rel_l2(sim.cpu().numpy(), rs) < 1e-5
    assert rel_l2(addon.cpu().numpy(), ra) < 1e-5
    assert rel_l2(conf.cpu().numpy(), rc) < 1e-5


def test_affine_ncc_and_gradient_match_oracle(pvr):
    cfg = synth.config_tiny(noise=True)
    geom = cfg["geom"]
    x = cfg["gt"].reshape(-1).astype(np.float32)
    desc, _ = synth.all_patches(geom, 32, 16)
    rng = np.random.default_rng(21)
    d = desc[rng.choice(desc.shape[0], 40, replace=False)].copy()
    off = 0
    for r in d:
        r[6] = off
        off += int(r[4] * r[5])
    y = synth.pack_patch_pixels(cfg["stacks"], d)
    poses = _affine(rng, len(d), dmax=0.06)
    ctx = _ctx(pvr, geom, dz=1.0)
    pt = pvr.PatchTable.from_numpy(d, off)
    ncc, grad = ctx.pvr_ncc_grad(_t(x), _t(y), pt, _t(poses))
    ncc, grad = ncc.cpu().numpy(), grad.cpu().numpy()
    assert grad.shape == (len(d), 12)
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 1.0)
    n_ok = 0
    for s in range(len(d)):
        rn, rg = O.ncc_grad(G, ps, x, y, d[s], poses[s], n_params=12)
        assert abs(ncc[s] - rn) < 2e-5, (s, ncc[s], rn)
        if rn != 0.0:
            n_ok += 1
            assert np.linalg.norm(grad[s] - rg) <= 2e-3 * np.linalg.norm(rg) + 1e-9, (s, grad[s], rg)
    assert n_ok > 30


@pytest.mark.parametrize("case", ["uneven", "tiled"])
def test_affine_pose_grad_matches_oracle(pvr, case):
    geom, desc, npix, _, rng = CASES[case]()
    poses = _affine(rng, desc.shape[0], dmax=0.05)
    from scipy.ndimage import gaussian_filter
    nx, ny, nz = geom.vol_dims
    x = (500.0 + 2000.0 * gaussian_filter(rng.normal(size=(nz, ny, nx)), 1.5)).astype(np.float32).reshape(-1)
    r = rng.normal(size=npix).astype(np.float32)
    ctx = _ctx(pvr, geom)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    g = ctx.pvr_pose_grad(_t(x), _t(r), pt, _t(poses)).cpu().numpy()
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 0.8)
    nz_ = 0
    for s in range(desc.shape[0]):
        _, rg = O.sim_pose_vjp(G, ps, x, r.astype(np.float64), desc[s], poses[s], n_params=12, exact=True)
        if np.linalg.norm(rg) == 0.0:
            assert np.all(g[s] == 0.0)
            continue
        nz_ += 1
        assert np.linalg.norm(g[s] - rg) <= 2e-3 * np.linalg.norm(rg), (s, g[s], rg)
    assert nz_ >= desc.shape[0] // 2


def test_affine_registration_recovers_known_transform(pvr):
    """Noiseless data simulated at known affine poses (stretch / shear of a
    few per cent, as breathing motion makes): registration from perturbed
    poses reaches NCC > 0.9999 and the residual displacement at the patch
    corners falls below 0.05 mm."""
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
    rng = np.random.default_rng(14)
    th_true = _affine(rng, len(d), dmax=0.04, trans=1.0)
    ctx = _ctx(pvr, geom, dz=1.0, reg_delta_min=1e-5)
    pt = pvr.PatchTable.from_numpy(d, npix)
    y, _ = ctx.pvr_simulate(_t(x), pt, _t(th_true))
    start = th_true.copy()
    start[:, :3] += rng.uniform(-2, 2, (len(d), 3))
    start[:, 3:] += rng.uniform(-0.04, 0.04, (len(d), 9))
    pg = _t(start)
    _, ncc = ctx.pvr_register(_t(x), y, pt, pg, 400)
    got = pg.cpu().numpy()
    assert np.all(ncc.cpu().numpy() > 0.9999)
    for s in range(len(d)):
        S = np.asarray(geom.p2w[int(d[s, 0])])
        half = np.array([(d[s, 4] - 1) / 2.0, (d[s, 5] - 1) / 2.0])
        dD = (got[s, 3:] - th_true[s, 3:]).reshape(3, 3)
        for sx in (-1, 1):
            for sy in (-1, 1):
                u = S[:, 0] * sx * half[0] + S[:, 1] * sy * half[1]
                assert np.linalg.norm((got[s, :3] - th_true[s, :3]) + dD @ u) < 0.05, s


def test_affine_context_rejects_the_rigid_proposal(pvr):
    """The pose-proposal network predicts rigid corrections; an affine
    context refuses it with PVR_ERR_UNSUPPORTED before anything runs."""
    geom, desc, npix, _, rng = uneven_case()
    ctx = _ctx(pvr, geom)
    net = pvr.Net(batch_max=4, seed=1)
    net.reserve(64, npix)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    x = torch.zeros(geom.n_vox, dtype=torch.float32, device="cuda")
    y = torch.zeros(npix, dtype=torch.float32, device="cuda")
    poses = torch.zeros((desc.shape[0], 12), dtype=torch.float64, device="cuda")
    with pytest.raises(pvr.PvrError) as e:
        net.propose(ctx, x, y, pt, poses, [1.0] * 6)
    assert e.value.code == -6
