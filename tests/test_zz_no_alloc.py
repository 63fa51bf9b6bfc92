"""The allocation-free forward model (pvr_simulate_noalloc) against the
regular pvr_simulate.

pvr_simulate_noalloc exists for callers that cannot allocate device memory
(an application whose own allocator owns the device, or a loop that must not
allocate once running): its scratch is a fixed array inside the library.
This file is collected last on purpose.  It checks two calls in a row with
different patch tables and volumes -- so a result left in the shared array
by the first call cannot pass for the second -- against pvr_simulate at the
tolerance of the simulate parity tests (valid mask exact, relative L2
1e-5), and that a call above the patch limit is rejected."""
import numpy as np
import pytest
import torch

from tests.cases import rel_l2, tiled_case, uneven_case

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def test_noalloc_simulate_matches_simulate_twice():
    from paper_1611_07289_b300 import pvr
    for case in (tiled_case, uneven_case):
        geom, desc, npix, poses, rng = case()
        x = rng.uniform(0, 1000, geom.n_vox).astype(np.float32)
        prm = pvr.default_params(psf_dz=0.8, max_patches=4096, max_pixels=1 << 22,
                                 max_patch_side=256)
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
