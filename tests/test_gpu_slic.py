"""Superpixel patches on the GPU: the SLIC patch table and membership masks
bit-exact against the numpy reference (oracle/slic_ref.py), and the forward
model, adjoint and NCC of superpixel patches against the oracle with the
masks applied."""
import numpy as np
import pytest
import torch
from scipy.ndimage import gaussian_filter

from oracle import pvr_oracle as O
from oracle import slic_ref
from paper_1611_07289_b300 import synth
from tests.cases import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pvr():
    from paper_1611_07289_b300 import pvr as m
    return m


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _case(seed):
    rng = np.random.default_rng(seed)
    n = 24
    w2v, v2w = synth.volume_geometry((n, n, n), 1.0)
    p2w = [synth.stack_matrix(*synth.rot_zyx(*rng.uniform(-25, 25, 3)).T, 60, 50, 3, 0.35, 2.0) for _ in range(2)]
    geom = synth.Geometry((n, n, n), w2v, v2w, [(60, 50, 3)] * 2, p2w, [2.0, 2.0])
    stacks = [(500 + 400 * gaussian_filter(rng.normal(size=(3, 50, 60)), (0, 3, 3)) / 0.05).astype(np.float32)
              for _ in range(2)]
    stacks = [np.abs(s) for s in stacks]
    return geom, stacks, rng


@pytest.mark.parametrize("a,t,gamma,keep", [(12, 10.0, 3, 0.0), (10, 4.0, 5, 0.5)])
def test_slic_table_and_members_are_exact(pvr, a, t, gamma, keep):
    geom, stacks, rng = _case(1)
    ctx = pvr.Context(geom, pvr.default_params(max_patches=4096, max_pixels=1 << 22, max_patch_side=128,
                                               slic_a_min=8))
    pt, n = ctx.pvr_patches_build_slic(_t(synth.pack_stacks(stacks)), a, t, gamma, n_iter=6, fg_frac=0.3,
                                       keep_frac=keep)
    desc, member, npix = slic_ref.patches_build_slic(geom.stack_dims, stacks, a, t, gamma, n_iter=6, fg_frac=0.3,
                                                     keep_frac=keep)
    assert n == desc.shape[0] > 0 and pt.n_pix == npix
    assert np.array_equal(pt.desc.cpu().numpy(), desc)
    assert np.array_equal(pt.member[:npix].cpu().numpy(), member)


def test_superpixel_patches_through_the_model(pvr):
    geom, stacks, rng = _case(2)
    ctx = pvr.Context(geom, pvr.default_params(psf_dz=0.8, max_patches=4096, max_pixels=1 << 22,
                                               max_patch_side=128, slic_a_min=8))
    packed = _t(synth.pack_stacks(stacks))
    pt, n = ctx.pvr_patches_build_slic(packed, 12, 10.0, 3, n_iter=6)
    desc = pt.desc.cpu().numpy()
    member = pt.member[:pt.n_pix].cpu().numpy()
    y = ctx.pvr_patches_gather(packed, pt)
    poses = synth.random_poses(rng, pt.n, rot=4.0, trans=1.0)
    x = rng.uniform(0, 1000, geom.n_vox).astype(np.float32)
    sim, valid = ctx.pvr_simulate(_t(x), pt, _t(poses))
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 0.8)
    fix = O.pose_fixed(G, ps, desc, poses)
    rs, rv, _ = O.simulate(G, ps, x, desc, fix, pt.n_pix)
    rv = rv & member
    assert np.array_equal(valid.cpu().numpy(), rv) and rv.sum() < member.sum() + 1
    assert rel_l2(sim.cpu().numpy() * rv, rs * rv) < 1e-5
    r = rng.normal(size=pt.n_pix).astype(np.float32)
    a_, c_ = ctx.pvr_adjoint(pt, _t(poses), _t(r), None)
    ra, rc = O.adjoint(G, ps, desc, fix, r=r.astype(np.float64), w=member.astype(np.float64))
    assert rel_l2(a_.cpu().numpy(), ra) < 1e-5 and rel_l2(c_.cpu().numpy(), rc) < 1e-5
    ncc, grad = ctx.pvr_ncc_grad(_t(x), y, pt, _t(poses))
    ncc, grad = ncc.cpu().numpy(), grad.cpu().numpy()
    yn = y.cpu().numpy()
    for s in range(min(pt.n, 12)):
        rn, rg = O.ncc_grad(G, ps, x, yn, desc[s], poses[s], member=member)
        assert abs(ncc[s] - rn) < 2e-5, (s, ncc[s], rn)
        if rn != 0.0:
            assert np.linalg.norm(grad[s] - rg) <= 2e-3 * np.linalg.norm(rg) + 1e-9
