"""The first super-resolution pass of pvr_reconstruct_iter takes the forward
model of one-tile patches from the registration's NCC kernels (each keeps
the residual, valid flags and EM tile partials at the patch's best pose)
instead of simulating again.  Checked against the same iteration with
32-pixel super-resolution tiles, where the patches span several tiles and
the pass simulates as usual: same poses and patch masks, same volume and EM
weights up to float32 reduction order."""
import numpy as np
import pytest
import torch

from paper_1611_07289_b300 import synth
from tests.cases import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pvr():
    from paper_1611_07289_b300 import pvr as m
    return m


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("fixed,evals,n_sr", [(0, 4, 1), (0, 2, 2), (1, 3, 1)])
def test_reused_forward_model_matches_simulating_pass(pvr, fixed, evals, n_sr):
    cfg = synth.config_tiny()
    geom = cfg["geom"]
    prm = dict(reg_evals=evals, reg_fixed_step=fixed, reg_delta0=0.5, n_sr=n_sr, max_patches=4096,
               max_pixels=1 << 22, max_patch_side=64)
    packed = _t(synth.pack_stacks(cfg["stacks"]))
    rng = np.random.default_rng(3)
    out = []
    for tile in (0, 32):
        ctx = pvr.Context(geom, pvr.default_params(**prm))
        pt, n = ctx.pvr_patches_build(packed, 64, 32)
        assert n > 0 and int(pt.desc[:, 4].max()) == 64
        y = ctx.pvr_patches_gather(packed, pt)
        if tile:
            t, m, _ = ctx.pvr_plan(pt, tile=tile, mode=0)
            assert t == 32
        poses = _t(synth.random_poses(np.random.default_rng(3), pt.n, rot=3.0, trans=1.0))
        x = _t(np.random.default_rng(4).uniform(0, 1000, geom.n_vox).astype(np.float32)).reshape(ctx.vol_shape)
        st = pvr.new_state()
        mask = torch.ones(pt.n, dtype=torch.uint8, device="cuda")
        p = torch.empty(pt.n_pix, dtype=torch.float32, device="cuda")
        w = torch.empty(pt.n, dtype=torch.float32, device="cuda")
        ctx.pvr_reconstruct_iter(x, y, pt, poses, st, mask, p, w)
        ctx.pvr_device_status()
        out.append((x.cpu().numpy(), poses.cpu().numpy(), mask.cpu().numpy(), p.cpu().numpy(), w.cpu().numpy(),
                    st.cpu().numpy()))
    (x0, p0, m0, pp0, w0, s0), (x1, p1, m1, pp1, w1, s1) = out
    assert np.array_equal(p0, p1) and np.array_equal(m0, m1)
    assert rel_l2(x0, x1) < 1e-5 and rel_l2(pp0, pp1) < 1e-5
    # the patch posteriors sit in the tail of the p-bar mixture, where a
    # relative change d of p-bar changes ln w by about d p-bar |p-bar - mu| /
    # sigma^2 (hundreds of times d with sigma^2 at its 1e-4 floor); a second
    # pass starts from volumes that differ in the float reduction order of the
    # adjoint (~1e-7), so they get a looser bound
    assert rel_l2(w0, w1) < 1e-4
    assert np.allclose(s0, s1, rtol=1e-4, atol=1e-9)


def test_reused_forward_model_with_superpixel_patches(pvr):
    """Superpixel patches (membership masks, uneven boxes up to 64 pixels):
    the kept forward model honours the masks like the simulate kernel."""
    cfg = synth.config_tiny()
    geom = cfg["geom"]
    prm = dict(reg_evals=3, reg_delta0=0.5, n_sr=1, max_patches=4096, max_pixels=1 << 22, max_patch_side=64,
               slic_a_min=16)
    packed = _t(synth.pack_stacks(cfg["stacks"]))
    out = []
    for tile in (0, 32):
        ctx = pvr.Context(geom, pvr.default_params(**prm))
        pt, n = ctx.pvr_patches_build_slic(packed, 16, 10.0, 2, n_iter=4)
        assert n > 0 and pt.member is not None
        y = ctx.pvr_patches_gather(packed, pt)
        if tile:
            t, m, _ = ctx.pvr_plan(pt, tile=tile, mode=0)
            assert t == 32
        poses = _t(synth.random_poses(np.random.default_rng(5), pt.n, rot=2.0, trans=0.5))
        x = _t(np.random.default_rng(6).uniform(0, 1000, geom.n_vox).astype(np.float32)).reshape(ctx.vol_shape)
        st = pvr.new_state()
        mask = torch.ones(pt.n, dtype=torch.uint8, device="cuda")
        p = torch.empty(pt.n_pix, dtype=torch.float32, device="cuda")
        ctx.pvr_reconstruct_iter(x, y, pt, poses, st, mask, p, None)
        ctx.pvr_device_status()
        member = pt.member[:pt.n_pix].cpu().numpy()
        out.append((x.cpu().numpy(), poses.cpu().numpy(), mask.cpu().numpy(), p.cpu().numpy(), member))
    (x0, p0, m0, pp0, mb0), (x1, p1, m1, pp1, mb1) = out
    assert np.array_equal(mb0, mb1) and np.array_equal(p0, p1) and np.array_equal(m0, m1)
    assert np.all(pp0[mb0 == 0] == 0)   # pixels outside their superpixel carry no weight
    assert rel_l2(x0, x1) < 1e-5 and rel_l2(pp0, pp1) < 1e-5
