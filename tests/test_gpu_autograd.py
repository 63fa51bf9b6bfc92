"""The differentiable forward model on the GPU: pvr_pose_grad against the
oracle's pose vector-Jacobian product, the autograd Function against the
oracle (adjoint and pose gradient) and against central finite differences of
the GPU forward model, and plain L2 gradient descent on volume and poses on
the 128^3 / 4,128 x 48^2 workload."""
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


def _textured(geom, seed):
    from scipy.ndimage import gaussian_filter
    nx, ny, nz = geom.vol_dims
    v = gaussian_filter(np.random.default_rng(seed).normal(size=(nz, ny, nx)), 1.5)
    return (500.0 + 2000.0 * v).astype(np.float32).reshape(-1)


@pytest.mark.parametrize("case", ["uneven", "tiled"])
def test_pose_grad_matches_oracle(pvr, case):
    if case == "uneven":
        geom, desc, npix, poses, rng = uneven_case(8)
    else:
        geom, desc, npix, poses, rng = tiled_case(2)
    x = _textured(geom, 1)
    r = rng.normal(size=npix).astype(np.float32)
    ctx = pvr.Context(geom, pvr.default_params(psf_dz=0.8, max_patches=4096, max_pixels=1 << 22,
                                               max_patch_side=256))
    pt = pvr.PatchTable.from_numpy(desc, npix)
    g = ctx.pvr_pose_grad(_t(x), _t(r), pt, _t(poses)).cpu().numpy()
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 0.8)
    nz = 0
    for s in range(desc.shape[0]):
        _, rg = O.sim_pose_vjp(G, ps, x, r.astype(np.float64), desc[s], poses[s], exact=True)
        if np.linalg.norm(rg) == 0.0:
            assert np.all(g[s] == 0.0)
            continue
        nz += 1
        assert np.linalg.norm(g[s] - rg) <= 2e-3 * np.linalg.norm(rg), (s, g[s], rg)
    assert nz >= desc.shape[0] // 2


def _interior_case(seed):
    """Patches whose PSF samples stay inside the volume for small poses, so
    the forward model is a smooth function of the pose (a sample leaving the
    volume changes the normalisation discontinuously)."""
    rng = np.random.default_rng(seed)
    geom = synth.random_geometry(rng, n=32, n_stacks=2, W=40, H=40, K=5, pix=0.5, thick=2.0)
    desc, npix = synth.all_patches(geom, 16, 8)
    poses = synth.random_poses(rng, desc.shape[0], rot=2.0, trans=1.0)
    return geom, desc, npix, poses, rng


def test_autograd_matches_oracle_and_finite_differences(pvr):
    from paper_1611_07289_b300.autograd import simulate_patches
    geom, desc, npix, poses, rng = _interior_case(9)
    x_np = _textured(geom, 2)
    ctx = pvr.Context(geom, pvr.default_params(psf_dz=0.8, max_patches=4096, max_pixels=1 << 22,
                                               max_patch_side=64))
    pt = pvr.PatchTable.from_numpy(desc, npix)
    w = _t(rng.normal(size=npix).astype(np.float32))
    x = _t(x_np).reshape(geom.vol_dims[::-1]).requires_grad_(True)
    th = _t(poses).requires_grad_(True)
    sim, valid = simulate_patches(x, th, ctx, pt)
    (sim * w).sum().backward()
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 0.8)
    fix = O.pose_fixed(G, ps, desc, poses)
    ra, _ = O.adjoint(G, ps, desc, fix, r=w.cpu().numpy().astype(np.float64))
    assert rel_l2(x.grad.reshape(-1).cpu().numpy(), ra) < 1e-5
    gp = th.grad.cpu().numpy()
    for s in range(desc.shape[0]):
        _, rg = O.sim_pose_vjp(G, ps, x_np, w.cpu().numpy().astype(np.float64), desc[s], poses[s])
        assert np.linalg.norm(gp[s] - rg) <= 2e-3 * np.linalg.norm(rg) + 1e-9
    # central differences of the GPU forward model with h = 1e-3 in the
    # registration's scaled units (mm of motion at the patch edge: angles
    # times the patch half-diagonal in radians), so that every parameter
    # moves the samples by about 1e-3 voxel -- far above the 2^-20 voxel
    # quantum of the fixed-point lattice, which a step of 1e-3 degree (about
    # 7e-5 voxel here) is not.  A secant that crosses a trilinear cell face
    # (about 6e-3 of the samples at this step) sees the jump of the
    # piecewise-constant trilinear slope; relative to the gradient that
    # error scales as the inverse smoothness length of the volume, so this
    # check uses a smoother zero-mean texture (correlation length 3 voxels;
    # a mean offset would only add float32 rounding).
    half_diag = 0.5 * np.hypot(16 * 0.5, 16 * 0.5)
    hk = np.array([1e-3] * 3 + [1e-3 / (half_diag * np.pi / 180.0)] * 3)
    from scipy.ndimage import gaussian_filter
    nx_, ny_, nz_ = geom.vol_dims
    smooth = gaussian_filter(np.random.default_rng(3).normal(size=(nz_, ny_, nx_)), 3.0)
    x0 = _t((200.0 * smooth / smooth.std()).astype(np.float32))
    thd = th.detach().clone().requires_grad_(True)
    s_fd, _ = simulate_patches(x0, thd, ctx, pt)
    (s_fd * w).sum().backward()
    gp0 = thd.grad.cpu().numpy()

    def loss(p):
        s_, _ = ctx.pvr_simulate(x0, pt, p)
        return float((s_.double() * w.double()).sum())

    worst = 0.0
    for s in rng.choice(desc.shape[0], 6, replace=False):
        fd = np.zeros(6)
        for k in range(6):
            tp, tm = th.detach().clone(), th.detach().clone()
            tp[s, k] += hk[k]
            tm[s, k] -= hk[k]
            fd[k] = (loss(tp) - loss(tm)) / (2 * hk[k])
        sc = 1.0 / np.array([1.0] * 3 + [half_diag * np.pi / 180.0] * 3)   # per scaled unit
        worst = max(worst, np.linalg.norm((fd - gp0[s]) * sc) / np.linalg.norm(fd * sc))
    assert worst < 1e-2, worst
    # the volume gradient by differences at a few voxels (the model is linear
    # in x, so A^T w does not depend on the volume it is taken at)
    xd = x0
    for v in rng.choice(geom.n_vox, 5, replace=False):
        xp, xm = xd.clone().reshape(-1), xd.clone().reshape(-1)
        xp[v] += 1.0
        xm[v] -= 1.0
        sp_, _ = ctx.pvr_simulate(xp.reshape(xd.shape), pt, th.detach())
        sm_, _ = ctx.pvr_simulate(xm.reshape(xd.shape), pt, th.detach())
        fdv = float(((sp_.double() - sm_.double()) * w.double()).sum()) / 2.0
        gv = float(x.grad.reshape(-1)[v])
        assert abs(fdv - gv) <= 1e-3 * max(abs(gv), 1.0), (v, fdv, gv)


def test_l2_descent_on_volume_and_poses(pvr):
    """Plain gradient descent on L = 1/2 sum_valid (sim(x, poses) - y)^2 with
    the autograd gradients: the loss falls at every step, and the poses move
    toward the true ones."""
    from paper_1611_07289_b300.autograd import simulate_patches
    cfg = synth.config_diff()
    geom, desc, npix = cfg["geom"], cfg["desc"], cfg["n_pix"]
    ctx = pvr.Context(geom, pvr.default_params(psf_dz=1.0, max_patches=len(desc), max_pixels=npix,
                                               max_patch_side=48))
    pt = pvr.PatchTable.from_numpy(desc, npix)
    x_true = _t(cfg["gt"].astype(np.float32))
    th_true = torch.zeros((len(desc), 6), dtype=torch.float64, device="cuda")
    y, vy = ctx.pvr_simulate(x_true, pt, th_true)
    rng = np.random.default_rng(4)
    th = (th_true + _t(synth.random_poses(rng, len(desc), rot=1.0, trans=1.0))).requires_grad_(True)
    x = (x_true * 0.8).requires_grad_(True)
    _, conf = ctx.pvr_adjoint(pt, th_true)
    ax = 1.0 / float(conf.max())           # below 2 / ||A^T A|| (rows of A sum to 1)
    losses, perr = [], []
    for it in range(6):
        sim, valid = simulate_patches(x, th, ctx, pt)
        r = (sim - y) * valid.float()
        L = 0.5 * (r * r).sum()
        losses.append(float(L.detach()))
        perr.append(float((th.detach() - th_true).abs().mean()))
        x.grad = th.grad = None
        L.backward()
        with torch.no_grad():
            x -= ax * x.grad
            # per-patch step of 0.05 (mm or degree) along the normalised gradient
            g = th.grad
            th -= 0.05 * g / g.norm(dim=1, keepdim=True).clamp_min(1e-30)
    assert all(b < a for a, b in zip(losses, losses[1:])), losses
    assert perr[-1] < perr[0], perr
