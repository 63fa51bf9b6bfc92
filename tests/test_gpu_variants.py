"""Paper variants on the GPU: the rigidity map (PSF-integrated p * p-bar) and
the per-patch evaluation with the local DSSIM heat map, against the oracle
and their closed forms."""
import numpy as np
import pytest
import torch

from oracle import pvr_oracle as O
from tests.cases import rel_l2, tiled_case, uneven_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pvr():
    from paper_1611_07289_b300 import pvr as m
    return m


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _ctx(pvr, geom):
    return pvr.Context(geom, pvr.default_params(psf_dz=0.8, max_patches=4096, max_pixels=1 << 22,
                                               max_patch_side=256))


@pytest.mark.parametrize("case", ["uneven", "tiled"])
def test_rigidity_map(pvr, case):
    geom, desc, npix, poses, rng = (uneven_case(6) if case == "uneven" else tiled_case(3))
    ctx = _ctx(pvr, geom)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    P = _t(poses)
    # p = 1, p-bar = 1: the map is 1 wherever a sample reaches, else 0
    ones_p = torch.ones(npix, device="cuda")
    ones_b = torch.ones(pt.n, device="cuda")
    R1 = ctx.pvr_rigidity_map(pt, P, ones_p, ones_b).cpu().numpy().reshape(-1)
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 0.8)
    fix = O.pose_fixed(G, ps, desc, poses)
    _, conf = O.adjoint(G, ps, desc, fix)
    reached = conf > 1e-6
    assert reached.sum() > 0 and np.allclose(R1[reached], 1.0, atol=1e-5) and np.all(R1[~reached] == 0)
    # random p and p-bar against the oracle's A^T(p p-bar) / A^T 1
    p = rng.uniform(0, 1, npix).astype(np.float32)
    pb = rng.uniform(0, 1, pt.n).astype(np.float32)
    R = ctx.pvr_rigidity_map(pt, P, _t(p), _t(pb)).cpu().numpy().reshape(-1)
    rr = p.astype(np.float64) * np.repeat(pb.astype(np.float64), desc[:, 4] * desc[:, 5])
    addon, _ = O.adjoint(G, ps, desc, fix, r=rr)
    ref = np.where(reached, addon / np.where(reached, conf, 1.0), 0.0)
    assert rel_l2(R, ref) < 1e-5


def test_patch_metrics_and_dssim_map(pvr):
    geom, desc, npix, poses, rng = uneven_case(7)
    ctx = _ctx(pvr, geom)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    y = rng.uniform(100, 900, npix).astype(np.float32)
    s = (y + rng.normal(0, 60, npix)).astype(np.float32)
    valid = (rng.uniform(size=npix) > 0.1).astype(np.uint8)
    out, m = ctx.pvr_patch_metrics(_t(y), _t(s), _t(valid), pt, w=3)
    ro, rm = O.patch_metrics(y, s, valid, desc, 3)
    out, m = out.cpu().numpy(), m.cpu().numpy()
    finite = np.isfinite(ro[:, 0])
    assert np.allclose(out[finite], ro[finite], rtol=1e-9, atol=1e-9)
    assert np.allclose(m, rm, rtol=1e-5, atol=1e-6)
    # identical patches: SSIM 1, an empty heat map
    out2, m2 = ctx.pvr_patch_metrics(_t(y), _t(y), _t(valid), pt, w=2)
    has = np.array([valid[o:o + n].any() for o, n in zip(desc[:, 6], desc[:, 4] * desc[:, 5])])
    assert np.allclose(out2.cpu().numpy()[has, 2], 1.0) and float(m2.abs().max()) < 1e-6
