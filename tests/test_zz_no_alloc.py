"""The allocation-free forward model (pvr_simulate_noalloc) against the
regular pvr_simulate.

pvr_simulate_noalloc exists for callers that cannot allocate device memory
(an application whose own allocator owns the device, or a loop that must not
allocate once running): its scratch is a fixed array inside the library.
This file is collected last on purpose.  It checks calls in a row with
different patch tables, volumes and pose kinds -- the largest table first,
then smaller ones, so a row left in the shared array by an earlier call
cannot pass for a later one -- against pvr_simulate at the tolerance of the
simulate parity tests (valid mask exact, relative L2 1e-5); that the error
word of the shared array reports a non-finite pose through
pvr_noalloc_status (and is clear again afterwards); and that a call above
the patch limit is rejected."""
import numpy as np
import pytest
import torch

from tests.cases import rel_l2, tiled_case, uneven_case

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _check(pvr, geom, desc, npix, poses, x, n_params=6):
    prm = pvr.default_params(psf_dz=0.8, max_patches=4096, max_pixels=1 << 22, max_patch_side=256,
                             n_params=n_params)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    ctx = pvr.Context(geom, prm)
    ref_s, ref_v = ctx.pvr_simulate(_t(x), pt, _t(poses))
    sim = torch.full((npix,), -1.0, dtype=torch.float32, device="cuda")
    valid = torch.full((npix,), 7, dtype=torch.uint8, device="cuda")
    rc = pvr.pvr_simulate_noalloc(geom, prm, _t(x), pt, _t(poses), sim, valid)
    torch.cuda.synchronize()
    assert rc == 0
    assert torch.equal(valid, ref_v)
    assert rel_l2(sim.cpu().numpy(), ref_s.cpu().numpy()) < 1e-5
    ctx.close()
    return pt, prm


def test_noalloc_simulate_matches_simulate_in_a_row():
    from paper_1611_07289_b300 import pvr
    assert pvr.pvr_noalloc_status() == 0
    # 45 patches (rigid), then 6 large multi-tile patches, then 45 again with
    # affine poses: each later call must rewrite the rows it reads
    geom, desc, npix, poses, rng = uneven_case()
    x = rng.uniform(0, 1000, geom.n_vox).astype(np.float32)
    _check(pvr, geom, desc, npix, poses, x)
    g2, d2, n2, p2, r2 = tiled_case()
    assert d2.shape[0] < desc.shape[0]
    _check(pvr, g2, d2, n2, p2, r2.uniform(0, 1000, g2.n_vox).astype(np.float32))
    aff = np.concatenate([rng.uniform(-2, 2, (desc.shape[0], 3)),
                          rng.uniform(-0.1, 0.1, (desc.shape[0], 9))], 1)
    _check(pvr, geom, desc, npix, aff, x, n_params=12)
    assert pvr.pvr_noalloc_status() == 0


def test_noalloc_reports_a_non_finite_pose():
    from paper_1611_07289_b300 import pvr
    geom, desc, npix, poses, rng = uneven_case(seed=3)
    x = rng.uniform(0, 1000, geom.n_vox).astype(np.float32)
    poses = poses.copy()
    poses[2, 4] = np.nan
    prm = pvr.default_params(psf_dz=0.8, max_patch_side=256)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    sim = torch.zeros(npix, dtype=torch.float32, device="cuda")
    valid = torch.zeros(npix, dtype=torch.uint8, device="cuda")
    assert pvr.pvr_simulate_noalloc(geom, prm, _t(x), pt, _t(poses), sim, valid) == 0
    assert pvr.pvr_noalloc_status() == -3          # PVR_ERR_NUMERIC, then cleared
    assert pvr.pvr_noalloc_status() == 0
    # the patch with the NaN pose has no valid pixel; the others match pvr_simulate
    o, n = int(desc[2, 6]), int(desc[2, 4] * desc[2, 5])
    assert int(valid[o:o + n].sum()) == 0
    poses[2, 4] = 0.0
    _check(pvr, geom, desc, npix, poses, x)


def test_noalloc_rejects_too_many_patches():
    from paper_1611_07289_b300 import pvr
    geom, desc, npix, poses, rng = uneven_case()
    reps = 8192 // desc.shape[0] + 1
    big = np.concatenate([desc] * reps)
    pt = pvr.PatchTable.from_numpy(big, npix)
    prm = pvr.default_params(psf_dz=0.8, max_patch_side=256)
    x = torch.zeros(geom.n_vox, dtype=torch.float32, device="cuda")
    out = torch.zeros(npix, dtype=torch.float32, device="cuda")
    v = torch.zeros(npix, dtype=torch.uint8, device="cuda")
    p = torch.zeros((big.shape[0], 6), dtype=torch.float64, device="cuda")
    assert big.shape[0] > 8192
    assert pvr.pvr_simulate_noalloc(geom, prm, x, pt, p, out, v) == -1
