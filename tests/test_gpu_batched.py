"""Batched patches of uneven sizes: the per-slice-size patch table against the
oracle, planned launches (persistent work queue or one CTA per slot, 32- or
64-pixel tiles, tuned or forced) against unplanned ones and the oracle, and a
captured CUDA graph of a whole iteration against the direct call."""
import numpy as np
import pytest
import torch

from oracle import pvr_oracle as O
from paper_1611_07289_b300 import synth
from tests.cases import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pvr():
    from paper_1611_07289_b300 import pvr as m
    return m


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _uneven_sizes_case(seed):
    """24^3 volume, two oblique 140x140-pixel stacks of 3 slices, one patch
    side per slice from {32, 48, 64, 96, 128} with stride side / 2."""
    rng = np.random.default_rng(seed)
    n = 24
    w2v, v2w = synth.volume_geometry((n, n, n), 1.0)
    p2w = [synth.stack_matrix(*synth.rot_zyx(*rng.uniform(-30, 30, 3)).T, 140, 140, 3, 0.15, 2.0)
           for _ in range(2)]
    geom = synth.Geometry((n, n, n), w2v, v2w, [(140, 140, 3)] * 2, p2w, [2.0, 2.0])
    stacks = [rng.uniform(0, 1000, (3, 140, 140)).astype(np.float32) for _ in range(2)]
    sa = rng.choice(np.array([32, 48, 64, 96, 128], np.int32), 6).astype(np.int32)
    return geom, stacks, sa, (sa // 2).astype(np.int32), rng


def test_multi_size_table_and_gather_are_exact(pvr):
    geom, stacks, sa, ss, rng = _uneven_sizes_case(1)
    packed = synth.pack_stacks(stacks)
    ctx = pvr.Context(geom, pvr.default_params(max_patches=4096, max_pixels=1 << 22, max_patch_side=128))
    for fg, keep in ((0.0, 0.0), (0.5, 0.5)):
        pt, n = ctx.pvr_patches_build_sizes(_t(packed), sa, ss, fg, keep)
        ref, rn = O.patches_build_sizes(O.geom(geom), packed, sa, ss, fg, keep)
        assert n == ref.shape[0] > 0 and pt.n_pix == rn
        assert np.array_equal(pt.desc.cpu().numpy(), ref)
        y = ctx.pvr_patches_gather(_t(packed), pt)
        assert np.array_equal(y.cpu().numpy(), synth.pack_patch_pixels(stacks, ref))
    assert len(set(ref[:, 4].tolist())) > 1


@pytest.fixture(scope="module")
def planned(pvr):
    geom, stacks, sa, ss, rng = _uneven_sizes_case(2)
    packed = _t(synth.pack_stacks(stacks))
    ctx = pvr.Context(geom, pvr.default_params(psf_dz=0.8, max_patches=4096, max_pixels=1 << 22,
                                               max_patch_side=128))
    pt, n = ctx.pvr_patches_build_sizes(packed, sa, ss)
    y = ctx.pvr_patches_gather(packed, pt)
    poses = synth.random_poses(rng, pt.n, rot=3.0, trans=0.5)
    x = rng.uniform(0, 1000, geom.n_vox).astype(np.float32)
    return dict(geom=geom, ctx=ctx, pt=pt, y=y, poses=poses, x=x, rng=rng)


def test_planned_launches_match_unplanned_and_oracle(pvr, planned):
    ctx, pt, geom = planned["ctx"], planned["pt"], planned["geom"]
    X, P = _t(planned["x"]), _t(planned["poses"])
    r = _t(planned["rng"].normal(size=pt.n_pix).astype(np.float32))
    ctx.pvr_plan_clear()
    s0, v0 = ctx.pvr_simulate(X, pt, P)
    a0, c0 = ctx.pvr_adjoint(pt, P, r, None)
    desc = pt.desc.cpu().numpy()
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 0.8)
    fix = O.pose_fixed(G, ps, desc, planned["poses"])
    rs, rv, _ = O.simulate(G, ps, planned["x"], desc, fix, pt.n_pix)
    assert np.array_equal(v0.cpu().numpy(), rv) and rel_l2(s0.cpu().numpy(), rs) < 1e-5
    ra, rc = O.adjoint(G, ps, desc, fix, r=r.cpu().numpy().astype(np.float64))
    for tile, mode in ((64, 0), (64, 1), (32, 0), (32, 1)):
        t, m, n_items = ctx.pvr_plan(pt, tile=tile, mode=mode)
        assert (t, m) == (tile, mode)
        if mode == 1:
            sizes = desc[:, 4].astype(np.int64)
            assert n_items == int(np.sum(((sizes + tile - 1) // tile) ** 2))
        s1, v1 = ctx.pvr_simulate(X, pt, P)
        assert torch.equal(v1, v0) and torch.equal(s1, s0), (tile, mode)
        # float32 reductions in scheduling order: the adjoint's own tolerance
        a1, c1 = ctx.pvr_adjoint(pt, P, r, None)
        assert rel_l2(a1.cpu().numpy(), ra) < 1e-5 and rel_l2(c1.cpu().numpy(), rc) < 1e-5
    t, m, _ = ctx.pvr_plan(pt, X, planned["y"], P)            # tuned
    assert t in (32, 64) and m in (0, 1)
    ctx.pvr_plan_clear()
    assert ctx.pvr_plan_info() == (0, -1, 0)


def test_planned_patch_order_leaves_ncc_and_gradient_unchanged(pvr, planned):
    """pvr_plan also fixes the launch order of the table's patches (sorted by
    the 32^3-voxel block of their centre).  The NCC kernels write one sum per
    tile, so NCC and gradient are bit-identical with and without that order:
    for the whole table (multi-tile patches: the chunked kernels) and for its
    patches of at most 64 pixels (one tile each: the persistent fused
    kernel, which takes tiles from a counter in that order)."""
    ctx, pt, y = planned["ctx"], planned["pt"], planned["y"]
    X, P = _t(planned["x"]), _t(planned["poses"])
    desc = pt.desc.cpu().numpy()
    small = np.flatnonzero(desc[:, 4] <= 64)
    sub = pvr.PatchTable(pt.desc[_t(small)].contiguous(), pt.n_pix)
    assert pt.max_side > 64 and 0 < small.size < pt.n and sub.max_side <= 64
    for table, poses in ((pt, P), (sub, P[_t(small)].contiguous())):
        ctx.pvr_plan_clear()
        n0, g0 = ctx.pvr_ncc_grad(X, y, table, poses)
        m0, _ = ctx.pvr_ncc_grad(X, y, table, poses, want_grad=False)
        ctx.pvr_plan(table, tile=64, mode=0)
        n1, g1 = ctx.pvr_ncc_grad(X, y, table, poses)
        m1, _ = ctx.pvr_ncc_grad(X, y, table, poses, want_grad=False)
        assert torch.equal(n0, n1) and torch.equal(g0, g1) and torch.equal(m0, m1)
        assert torch.isfinite(g0).all() and (n0 != 0).any()
    ctx.pvr_plan_clear()


def _spatial_order(geom, desc):
    """The documented launch order: patches stably sorted by the 32^3-voxel
    block (z, then y, then x) holding their centre at the identity pose."""
    d = np.asarray(desc, dtype=np.int64)
    W = np.asarray(geom.w2v, dtype=np.float64)
    keys = np.zeros(len(d), dtype=np.int64)
    for i, row in enumerate(d):
        P = np.asarray(geom.p2w[row[0]], dtype=np.float64)
        ci, cj, k = row[2] + 0.5 * row[4] - 0.5, row[3] + 0.5 * row[5] - 0.5, float(row[1])
        w = [P[r, 0] * ci + P[r, 1] * cj + P[r, 2] * k + P[r, 3] for r in range(3)]
        b = []
        for r in range(3):
            v = W[r, 0] * w[0] + W[r, 1] * w[1] + W[r, 2] * w[2] + W[r, 3]
            b.append(int(v / 32.0) if 0.0 <= v < 32.0 * 1023.0 else (1023 if v >= 0.0 else 0))
        keys[i] = (b[2] * 1024 + b[1]) * 1024 + b[0]
    return np.argsort(keys, kind="stable").astype(np.int32), keys


def test_plan_order_is_the_spatial_sort(pvr):
    """pvr_plan_order returns a permutation equal to the documented sort of
    the 128^3 workload's 4,128 patches (three stacks, many 32^3 blocks)."""
    cfg = synth.config_diff()
    geom, desc, npix = cfg["geom"], cfg["desc"], cfg["n_pix"]
    ctx = pvr.Context(geom, pvr.default_params(max_patches=len(desc), max_pixels=npix, max_patch_side=48))
    pt = pvr.PatchTable.from_numpy(desc, npix)
    with pytest.raises(pvr.PvrError):
        ctx.pvr_plan_order(pt.n)                      # no plan yet
    ctx.pvr_plan(pt, tile=64, mode=0)
    order = ctx.pvr_plan_order(pt.n)
    ref, keys = _spatial_order(geom, desc)
    assert len(np.unique(keys)) > 20
    assert np.array_equal(np.sort(order), np.arange(pt.n))
    assert np.array_equal(order, ref)
    with pytest.raises(pvr.PvrError):
        ctx.pvr_plan_order(pt.n - 1)                  # another count
    ctx.pvr_plan_clear()
    ctx.close()


def test_iteration_plan_and_graph_match_direct_call(pvr, planned):
    ctx, pt = planned["ctx"], planned["pt"]
    y = planned["y"]

    def fresh():
        x = _t(planned["x"]).reshape(ctx.vol_shape).clone()
        return (x, _t(planned["poses"]).clone(), pvr.new_state(),
                torch.ones(pt.n, dtype=torch.uint8, device="cuda"))

    ctx.pvr_plan_clear()
    x0, p0, st0, m0 = fresh()
    ctx.pvr_reconstruct_iter(x0, y, pt, p0, st0, m0)
    ctx.pvr_plan(pt, _t(planned["x"]), y, _t(planned["poses"]))
    x1, p1, st1, m1 = fresh()
    ctx.pvr_reconstruct_iter(x1, y, pt, p1, st1, m1)
    assert torch.equal(p1, p0) and torch.equal(m1, m0)
    assert rel_l2(x1.cpu().numpy(), x0.cpu().numpy()) < 1e-5
    s = torch.cuda.Stream()
    x2, p2, st2, m2 = fresh()
    ctx.pvr_graph_capture(x2, y, pt, p2, st2, m2, stream=s)
    s.synchronize()
    assert torch.equal(x2.reshape(-1), _t(planned["x"]))     # capture runs nothing
    # calls on one context must not overlap on the GPU: order s after the
    # default stream's work (torch streams do not wait for it by themselves)
    s.wait_stream(torch.cuda.current_stream())
    ctx.pvr_graph_launch(stream=s)
    s.synchronize()
    assert torch.equal(p2, p0) and torch.equal(m2, m0)
    assert rel_l2(x2.cpu().numpy(), x0.cpu().numpy()) < 1e-5
    # a second replay continues from the updated state, like a direct call
    # from copies of that state (same inputs: the registration decisions
    # agree, only the adjoint's reduction order differs)
    x3, p3, st3, m3 = x2.clone(), p2.clone(), st2.clone(), m2.clone()
    ctx.pvr_reconstruct_iter(x3, y, pt, p3, st3, m3)
    s.wait_stream(torch.cuda.current_stream())
    ctx.pvr_graph_launch(stream=s)
    s.synchronize()
    assert torch.equal(p2, p3) and torch.equal(m2, m3)
    assert rel_l2(x2.cpu().numpy(), x3.cpu().numpy()) < 1e-5
    ctx.pvr_plan_clear()
