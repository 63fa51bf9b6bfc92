"""Parity at the benchmark's full size (uterus workload: 256x256x192 volume,
4 x 96 x 256^2 stacks, patches 64 / stride 32, about 18k patches and 74M
patch-pixels) in the launch configuration bench.py times (context with
max_patch_side 64: one 64x64 tile per CTA; the launch plan the benchmark's
tuner picks for this table, 64-pixel tiles with one CTA per tile, which also
fixes the spatial patch launch order).

The oracle cannot process 74M patch-pixels in seconds, so it is compared on
sampled patches of the full-size GPU outputs (forward model, NCC and its
gradient), on the full patch table and lattice (cheap and bit-exact), on
sampled rows of the adjoint scattered over the full grid (element by
element, every stack: the axial, coronal and sagittal ones and the oblique
30-degree one), and through properties that hold at any size (the
adjoint's dot-product test, the EM statistics on the full pixel set).  The
affine lattice and NCC gradient are checked the same way."""
import numpy as np
import pytest
import torch

from oracle import pvr_oracle as O
from paper_1611_07289_b300 import synth
from tests.cases import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    from paper_1611_07289_b300 import pvr
    cfg = synth.config_uterus(device="cuda")
    geom = cfg["geom"]
    packed_np = synth.pack_stacks(cfg["stacks"])
    packed = torch.as_tensor(packed_np, device="cuda")
    prm = pvr.default_params(psf_dz=0.75, max_patches=32768, max_pixels=1 << 27, max_patch_side=64)
    ctx = pvr.Context(geom, prm)
    pt, n = ctx.pvr_patches_build(packed, 64, 32, 0.01, 0.5)
    y = ctx.pvr_patches_gather(packed, pt)
    assert ctx.pvr_plan(pt, tile=64, mode=0)[:2] == (64, 0)
    rng = np.random.default_rng(7289)
    poses = synth.random_poses(rng, pt.n, rot=5.0, trans=3.0)
    return dict(pvr=pvr, cfg=cfg, geom=geom, packed_np=packed_np, ctx=ctx, pt=pt, n=n, y=y,
                poses=poses, rng=rng, G=O.geom(geom), ps=O.psf(1.2, 1, 3, 0.75))


def _sample(desc, y_np, idx):
    d = desc[idx].copy()
    ys, off = [], 0
    for r in d:
        n = int(r[4] * r[5])
        ys.append(y_np[int(r[6]):int(r[6]) + n])
        r[6] = off
        off += n
    return d, np.concatenate(ys), off


def test_full_patch_table_and_lattice_bit_exact(full):
    desc = full["pt"].desc.cpu().numpy()
    ref, npix = O.patches_build(full["G"], full["packed_np"], 64, 32, 0.01, 0.5)
    assert desc.shape[0] == full["n"] == ref.shape[0] > 5000
    assert np.array_equal(desc, ref) and full["pt"].n_pix == npix
    assert np.array_equal(full["y"].cpu().numpy(), synth.pack_patch_pixels(full["cfg"]["stacks"], ref))
    fix = full["ctx"].pvr_pose_to_fixed(full["pt"], torch.as_tensor(full["poses"], device="cuda"))
    rfix = O.pose_fixed(full["G"], full["ps"], ref, full["poses"])
    assert np.array_equal(fix.cpu().numpy()[:, :13].astype(np.int64), rfix[:, :13])


def test_full_simulate_sampled_patches(full):
    ctx, pt = full["ctx"], full["pt"]
    x = full["rng"].uniform(0, 1000, full["geom"].n_vox).astype(np.float32)
    sim, valid = ctx.pvr_simulate(torch.as_tensor(x, device="cuda"), pt,
                                  torch.as_tensor(full["poses"], device="cuda"))
    sim, valid = sim.cpu().numpy(), valid.cpu().numpy()
    desc = pt.desc.cpu().numpy()
    idx = np.sort(full["rng"].choice(desc.shape[0], 24, replace=False))
    d, _, npix = _sample(desc, np.zeros(pt.n_pix, np.float32), idx)
    fix = O.pose_fixed(full["G"], full["ps"], d, full["poses"][idx])
    rs, rv, _ = O.simulate(full["G"], full["ps"], x, d, fix, npix)
    gs, gv = _sample(desc, sim, idx)[1], _sample(desc, valid, idx)[1]
    assert np.array_equal(gv, rv)
    assert rel_l2(gs, rs) < 1e-5


def test_full_adjoint_dot_product(full):
    ctx, pt = full["ctx"], full["pt"]
    rng = np.random.default_rng(11)
    x = rng.normal(size=full["geom"].n_vox).astype(np.float32)
    r = rng.normal(size=pt.n_pix).astype(np.float32)
    P = torch.as_tensor(full["poses"], device="cuda")
    ax, _ = ctx.pvr_simulate(torch.as_tensor(x, device="cuda"), pt, P)
    atr, conf = ctx.pvr_adjoint(pt, P, torch.as_tensor(r, device="cuda"), None)
    lhs = float(torch.dot(ax.double(), torch.as_tensor(r, device="cuda").double()))
    rhs = float(torch.dot(torch.as_tensor(x, device="cuda").double(), atr.reshape(-1).double()))
    assert abs(lhs - rhs) / (float(ax.double().norm()) * float(np.linalg.norm(r))) < 1e-5
    # conf = A^T 1 restricted to valid pixels: its total is the number of valid pixels
    _, valid = ctx.pvr_simulate(torch.as_tensor(x, device="cuda"), pt, P)
    assert abs(float(conf.double().sum()) - float(valid.double().sum())) < 1e-4 * float(valid.double().sum())


def test_full_adjoint_sampled_rows_elementwise(full):
    """pvr_adjoint of 24 sampled rows (6 per stack) at the full volume size,
    element by element against the oracle over all 12.6 M voxels: the
    sagittal stack runs the through-plane (zeta) lane order of the scatter,
    the others the lattice orders, and the oblique stack crosses cell faces
    along all three axes."""
    ctx, pt = full["ctx"], full["pt"]
    desc = pt.desc.cpu().numpy()
    rng = np.random.default_rng(31)
    stacks = np.unique(desc[:, 0])
    assert len(stacks) == 4
    idx = np.sort(np.concatenate([rng.choice(np.flatnonzero(desc[:, 0] == s), 6, replace=False)
                                  for s in stacks]))
    d, _, npix = _sample(desc, np.zeros(pt.n_pix, np.float32), idx)
    poses = full["poses"][idx]
    r = rng.normal(size=npix).astype(np.float32)
    w = rng.uniform(0.2, 1.0, npix).astype(np.float32)
    sub = full["pvr"].PatchTable.from_numpy(d, npix)
    addon, conf = ctx.pvr_adjoint(sub, torch.as_tensor(poses, device="cuda"),
                                  torch.as_tensor(r, device="cuda"), torch.as_tensor(w, device="cuda"))
    fix = O.pose_fixed(full["G"], full["ps"], d, poses)
    ra, rc = O.adjoint(full["G"], full["ps"], d, fix, r=r.astype(np.float64), w=w.astype(np.float64))
    ga, gc = addon.cpu().numpy().reshape(-1), conf.cpu().numpy().reshape(-1)
    assert np.count_nonzero(rc) > 24 * 4096
    # the same voxels are reached, and the values agree
    assert np.array_equal(gc > 0, rc > 0)
    assert rel_l2(ga, ra) < 1e-5 and rel_l2(gc, rc) < 1e-5
    # per stack as well (each stack's rows alone)
    for s in stacks:
        rows = np.flatnonzero(d[:, 0] == s)
        ds, _, nps = _sample(d, np.zeros(npix, np.float32), rows)
        pix = np.concatenate([np.arange(int(d[k, 6]), int(d[k, 6]) + int(d[k, 4] * d[k, 5])) for k in rows])
        a1, c1 = ctx.pvr_adjoint(full["pvr"].PatchTable.from_numpy(ds, nps), torch.as_tensor(poses[rows], device="cuda"),
                                 torch.as_tensor(r[pix], device="cuda"), torch.as_tensor(w[pix], device="cuda"))
        f1 = O.pose_fixed(full["G"], full["ps"], ds, poses[rows])
        ra1, rc1 = O.adjoint(full["G"], full["ps"], ds, f1, r=r[pix].astype(np.float64), w=w[pix].astype(np.float64))
        assert rel_l2(a1.cpu().numpy(), ra1) < 1e-5 and rel_l2(c1.cpu().numpy(), rc1) < 1e-5, s


def test_full_affine_lattice_and_ncc_gradient(full):
    """Affine poses (12 parameters, breathing-like stretch and shear) at full
    size: the lattice of all patches bit-exact, NCC and gradient on sampled
    patches."""
    pvr = full["pvr"]
    prm = pvr.default_params(psf_dz=0.75, max_patches=32768, max_pixels=1 << 27, max_patch_side=64,
                             n_params=12)
    ctx = pvr.Context(full["geom"], prm)
    pt = full["pt"]
    rng = np.random.default_rng(41)
    poses = np.concatenate([rng.uniform(-3, 3, (pt.n, 3)), rng.uniform(-0.05, 0.05, (pt.n, 9))], 1)
    P = torch.as_tensor(poses, device="cuda")
    desc = pt.desc.cpu().numpy()
    fix = ctx.pvr_pose_to_fixed(pt, P)
    rfix = O.pose_fixed(full["G"], full["ps"], desc, poses, n_params=12)
    assert np.array_equal(fix.cpu().numpy()[:, :13].astype(np.int64), rfix[:, :13])
    x = full["cfg"]["gt"].reshape(-1).astype(np.float32)
    ncc, grad = ctx.pvr_ncc_grad(torch.as_tensor(x, device="cuda"), full["y"], pt, P)
    ncc, grad = ncc.cpu().numpy(), grad.cpu().numpy()
    y_np = full["y"].cpu().numpy()
    idx = np.sort(rng.choice(desc.shape[0], 12, replace=False))
    d, ys, _ = _sample(desc, y_np, idx)
    for k, s in enumerate(idx):
        rn, rg = O.ncc_grad(full["G"], full["ps"], x, ys, d[k], poses[s], n_params=12)
        assert abs(ncc[s] - rn) < 2e-5, (s, ncc[s], rn)
        if rn != 0.0:
            assert np.linalg.norm(grad[s] - rg) <= 2e-3 * np.linalg.norm(rg) + 1e-9, (s, grad[s], rg)
    ctx.close()


def test_full_ncc_gradient_sampled_patches(full):
    ctx, pt = full["ctx"], full["pt"]
    x = full["cfg"]["gt"].reshape(-1).astype(np.float32)
    P = torch.as_tensor(full["poses"], device="cuda")
    ncc, grad = ctx.pvr_ncc_grad(torch.as_tensor(x, device="cuda"), full["y"], pt, P)
    ncc, grad = ncc.cpu().numpy(), grad.cpu().numpy()
    desc = pt.desc.cpu().numpy()
    y_np = full["y"].cpu().numpy()
    idx = np.sort(full["rng"].choice(desc.shape[0], 12, replace=False))
    d, ys, _ = _sample(desc, y_np, idx)
    for k, s in enumerate(idx):
        rn, rg = O.ncc_grad(full["G"], full["ps"], x, ys, d[k], full["poses"][s])
        assert abs(ncc[s] - rn) < 2e-5, (s, ncc[s], rn)
        if rn != 0.0:
            assert np.linalg.norm(grad[s] - rg) <= 2e-3 * np.linalg.norm(rg) + 1e-9, (s, grad[s], rg)


def test_full_em_statistics(full):
    ctx, pt = full["ctx"], full["pt"]
    pvr = full["pvr"]
    rng = np.random.default_rng(12)
    y = full["y"].cpu().numpy()
    sim = (y + rng.normal(0, 15, y.size)).astype(np.float32)
    desc = pt.desc.cpu().numpy()
    for b in rng.choice(desc.shape[0], desc.shape[0] // 20, replace=False):   # outlier patches
        o, n = int(desc[b, 6]), int(desc[b, 4] * desc[b, 5])
        sim[o:o + n] += rng.normal(0, 150, n).astype(np.float32)
    valid = (rng.uniform(size=y.size) > 0.02).astype(np.uint8)
    st = pvr.new_state()
    p, wp, pb, mo = ctx.pvr_em_weights(full["y"], torch.as_tensor(sim, device="cuda"),
                                       torch.as_tensor(valid, device="cuda"), pt, st)
    sto = O.new_state()
    rp, rwp, rpb, rmo = O.em_weights(y, sim.astype(np.float64), valid, desc, O.em_params(), sto)
    sg = st.cpu().numpy()
    for k in ("SIGMA2", "C", "M", "MU_P", "SIGMA2_P", "C_P"):
        i = O.ST[k]
        assert abs(sg[i] - sto[i]) <= 1e-5 * max(abs(sto[i]), 1e-12), (k, sg[i], sto[i])
    assert rel_l2(p.cpu().numpy(), rp) < 1e-5
    assert rel_l2(pb.cpu().numpy(), rpb) < 1e-5
    near = np.abs(rwp - 0.5) < 1e-4
    assert np.array_equal(mo.cpu().numpy()[~near], rmo[~near])
