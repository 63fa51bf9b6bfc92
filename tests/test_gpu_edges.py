"""Edge cases of the C ABI on the GPU: empty tables, patches entirely
outside the volume, malformed patch rows and non-finite poses (reported by
the device error word, nothing written for the row), host-side argument
errors, degenerate NCC, constant residuals in EM, the largest patch side
and the largest PSF support."""
import numpy as np
import pytest
import torch

from oracle import pvr_oracle as O
from paper_1611_07289_b300 import synth
from tests.cases import rel_l2, uneven_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pvr():
    from paper_1611_07289_b300 import pvr as m
    return m


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _ctx(pvr, geom, **kw):
    base = dict(psf_dz=0.8, max_patches=4096, max_pixels=1 << 22, max_patch_side=256)
    base.update(kw)
    return pvr.Context(geom, pvr.default_params(**base))


def test_empty_patch_table_is_a_no_op(pvr):
    geom, desc, npix, poses, rng = uneven_case()
    ctx = _ctx(pvr, geom)
    empty = pvr.PatchTable(torch.zeros((0, 8), dtype=torch.int32, device="cuda"), 0, 1)
    x = torch.ones(geom.n_vox, device="cuda")
    p0 = torch.zeros((0, 6), dtype=torch.float64, device="cuda")
    sim = torch.zeros(1, device="cuda")
    v = torch.zeros(1, dtype=torch.uint8, device="cuda")
    ctx.pvr_simulate(x, empty, p0, sim, v)
    a, c = ctx.pvr_adjoint(empty, p0)
    assert float(a.abs().sum()) == 0.0 and float(c.abs().sum()) == 0.0
    ncc, _ = ctx.pvr_ncc_grad(x, sim, empty, p0)
    ctx.pvr_register(x, sim, empty, p0, 3)
    ctx.pvr_device_status()


def test_patch_outside_the_volume_is_invalid(pvr):
    geom, desc, npix, poses, rng = uneven_case(2)
    poses = poses.copy()
    poses[0, :3] = [400.0, 0.0, 0.0]       # 40 cm away: every sample outside
    poses[1, :3] = [5.0e3, 0.0, 0.0]       # beyond the fixed-point range: patch empty
    ctx = _ctx(pvr, geom)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    x = rng.uniform(0, 1, geom.n_vox).astype(np.float32)
    sim, valid = ctx.pvr_simulate(_t(x), pt, _t(poses))
    sim, valid = sim.cpu().numpy(), valid.cpu().numpy()
    for s in (0, 1):
        o, n = desc[s, 6], desc[s, 4] * desc[s, 5]
        assert np.all(valid[o:o + n] == 0) and np.all(sim[o:o + n] == 0)
    fix = ctx.pvr_pose_to_fixed(pt, _t(poses)).cpu().numpy()
    assert fix[1, 12] == 0 and fix[0, 12] == 1
    ctx.pvr_device_status()


def test_malformed_row_and_nan_pose_are_reported_and_skipped(pvr):
    geom, desc, npix, poses, rng = uneven_case(3)
    bad = desc.copy()
    bad[0, 2] = geom.stack_dims[bad[0, 0]][0]      # x0 = W: the row leaves its stack
    ctx = _ctx(pvr, geom)
    pt = pvr.PatchTable.from_numpy(bad, npix)
    x = _t(rng.uniform(0, 1, geom.n_vox).astype(np.float32))
    sim = torch.full((npix,), -7.0, device="cuda")
    valid = torch.full((npix,), 9, dtype=torch.uint8, device="cuda")
    ctx.pvr_simulate(x, pt, _t(poses), sim, valid)
    with pytest.raises(pvr.PvrError) as ei:
        ctx.pvr_device_status()
    assert ei.value.code == -4
    o, n = desc[0, 6], desc[0, 4] * desc[0, 5]
    assert torch.all(sim[o:o + n] == -7.0) and torch.all(valid[o:o + n] == 9)   # untouched
    assert not torch.any(sim[o + n:] == -7.0)
    ctx.pvr_device_status()                          # the word was cleared
    nanp = poses.copy()
    nanp[2, 4] = np.nan
    pt2 = pvr.PatchTable.from_numpy(desc, npix)
    sim2, valid2 = ctx.pvr_simulate(x, pt2, _t(nanp))
    with pytest.raises(pvr.PvrError) as ei:
        ctx.pvr_device_status()
    assert ei.value.code == -3
    o, n = desc[2, 6], desc[2, 4] * desc[2, 5]
    assert torch.all(valid2[o:o + n] == 0)


def test_host_argument_errors(pvr):
    geom, desc, npix, poses, rng = uneven_case(4)
    ctx = _ctx(pvr, geom, max_patches=8, max_patch_side=16)
    big = pvr.PatchTable.from_numpy(np.concatenate([desc] * 2), npix)
    x = torch.zeros(geom.n_vox, device="cuda")
    with pytest.raises(pvr.PvrError) as ei:
        ctx.pvr_simulate(x, big, torch.zeros((big.n, 6), dtype=torch.float64, device="cuda"))
    assert ei.value.code == -1 and "patch count" in str(ei.value)
    small = pvr.PatchTable(_t(desc[:4]), npix, max_side=33)
    with pytest.raises(pvr.PvrError) as ei:
        ctx.pvr_simulate(x, small, _t(poses[:4]))      # max side above the context's 16
    assert "max_side" in str(ei.value)
    ctx2 = _ctx(pvr, geom)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    m = torch.ones(pt.n, dtype=torch.uint8, device="cuda")
    y = torch.zeros(npix, device="cuda")
    with pytest.raises(pvr.PvrError):
        ctx2.pvr_em_weights(y, y, torch.ones(npix, dtype=torch.uint8, device="cuda"), pt,
                            pvr.new_state(), mask_in=m, mask_out=m)


def test_degenerate_ncc_and_constant_residuals(pvr):
    geom, desc, npix, poses, rng = uneven_case(5)
    ctx = _ctx(pvr, geom)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    x = _t(rng.uniform(0, 1, geom.n_vox).astype(np.float32))
    y = torch.full((npix,), 3.0, device="cuda")      # constant patches: NCC undefined
    P = _t(poses)
    ncc, grad = ctx.pvr_ncc_grad(x, y, pt, P)
    assert float(ncc.abs().max()) == 0.0 and float(grad.abs().max()) == 0.0
    P2 = P.clone()
    ctx.pvr_register(x, y, pt, P2, 5)
    assert torch.equal(P2, P)                         # no update
    sim = torch.zeros(npix, device="cuda")
    valid = torch.ones(npix, dtype=torch.uint8, device="cuda")
    st = pvr.new_state()
    p, wp, pb, mo = ctx.pvr_em_weights(y, sim, valid, pt, st)
    assert float(st[pvr.ST["M"]]) == 0.0 and torch.all(p == 1.0)


@pytest.mark.parametrize("kxy,kz,side", [(3, 8, 40), (1, 3, 256)])
def test_largest_support_and_patch_side(pvr, kxy, kz, side):
    rng = np.random.default_rng(13)
    n = 24
    w2v, v2w = synth.volume_geometry((n, n, n), 1.0)
    p2w = [synth.stack_matrix(*synth.rot_zyx(*rng.uniform(-20, 20, 3)).T, 260, 260, 3, 0.08, 1.5)]
    geom = synth.Geometry((n, n, n), w2v, v2w, [(260, 260, 3)], p2w, [1.5])
    desc = np.array([[0, 1, 2, 3, side, side, 0, 0]], dtype=np.int32)
    npix = side * side
    poses = synth.random_poses(rng, 1, rot=4.0, trans=0.5)
    x = rng.uniform(0, 1000, geom.n_vox).astype(np.float32)
    ctx = pvr.Context(geom, pvr.default_params(psf_kxy=kxy, psf_kz=kz, psf_dz=0.3, max_patches=16,
                                                max_pixels=1 << 17, max_patch_side=256))
    pt = pvr.PatchTable.from_numpy(desc, npix)
    sim, valid = ctx.pvr_simulate(_t(x), pt, _t(poses))
    G, ps = O.geom(geom), O.psf(1.2, kxy, kz, 0.3)
    fix = O.pose_fixed(G, ps, desc, poses)
    rs, rv, _ = O.simulate(G, ps, x, desc, fix, npix)
    assert np.array_equal(valid.cpu().numpy(), rv) and rv.sum() > 0
    assert rel_l2(sim.cpu().numpy(), rs) < 1e-5
    r = rng.normal(size=npix).astype(np.float32)
    a, c = ctx.pvr_adjoint(pt, _t(poses), _t(r), None)
    ra, rc = O.adjoint(G, ps, desc, fix, r=r.astype(np.float64))
    assert rel_l2(a.cpu().numpy(), ra) < 1e-5 and rel_l2(c.cpu().numpy(), rc) < 1e-5
