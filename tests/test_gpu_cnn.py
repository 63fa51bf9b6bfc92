"""The pose-proposal CNN on the tensor cores against a plain PyTorch CPU
reference (oracle/cnn_ref.py) that rounds to bfloat16 where the GPU stores
bfloat16: forward outputs, the loss, every parameter gradient, and that a
few Adam steps on a fixed batch lower the loss."""
import numpy as np
import pytest
import torch

from oracle import cnn_ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pvr():
    from paper_1611_07289_b300 import pvr as m
    return m


def _batch(rng, B):
    desc = np.array([[0, 0, 0, 0, 64, 64, 4096 * b, 0] for b in range(B)], dtype=np.int32)
    npix = 4096 * B
    yy, xx = np.meshgrid(np.arange(64), np.arange(64), indexing="ij")
    y = np.zeros(npix, np.float32)
    s = np.zeros(npix, np.float32)
    for b in range(B):
        cx, cy, r = rng.uniform(16, 48, 2).tolist() + [rng.uniform(6, 20)]
        img = 300 + 500 * (((xx - cx) ** 2 + (yy - cy) ** 2) < r * r) + rng.normal(0, 20, (64, 64))
        sh = rng.integers(-4, 5, 2)
        y[4096 * b:4096 * (b + 1)] = img.reshape(-1)
        s[4096 * b:4096 * (b + 1)] = np.roll(img, tuple(sh), axis=(0, 1)).reshape(-1)
    valid = (rng.uniform(size=npix) > 0.05).astype(np.uint8)
    target = rng.normal(0, 1, (B, 6)).astype(np.float32)
    return desc, npix, y, s, valid, target


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def test_cnn_forward_and_gradients_match_reference(pvr):
    rng = np.random.default_rng(0)
    B = 6
    desc, npix, y, s, valid, target = _batch(rng, B)
    net = pvr.Net(batch_max=8, seed=3)
    flat = net.get_params()
    assert flat.size == net.param_count() == sum(co * 9 * ci + co for ci, co, _ in cnn_ref.LAYERS) + 6 * cnn_ref.FEAT + 6
    pt = pvr.PatchTable.from_numpy(desc, npix)
    dev = lambda a: torch.as_tensor(a, device="cuda")
    out = net.forward(dev(y), dev(s), dev(valid), pt).cpu().numpy()
    img = cnn_ref.inputs(y, s, valid, desc)
    loss_r, out_r, g_r = cnn_ref.loss_and_grads(flat, img, target)
    assert _rel(out, out_r) < 1e-2, (out, out_r)
    loss = torch.zeros(1, device="cuda")
    net.train_step(dev(y), dev(s), dev(valid), pt, 0, B, dev(target), 1e-12, loss)
    assert abs(float(loss) - loss_r) < 1e-2 * loss_r
    g = net.get_grads()
    o = 0
    for ci, co, _ in cnn_ref.LAYERS:
        n = co * 9 * ci
        gw, gb = g[o:o + n], g[o + n:o + n + co]
        rw, rb = g_r[o:o + n], g_r[o + n:o + n + co]
        assert _rel(gw, rw) < 3e-2 and _rel(gb, rb) < 3e-2, (ci, co, _rel(gw, rw), _rel(gb, rb))
        o += n + co
    assert _rel(g[o:], g_r[o:]) < 1e-2


def test_cnn_training_lowers_the_loss(pvr):
    rng = np.random.default_rng(1)
    B = 8
    desc, npix, y, s, valid, target = _batch(rng, B)
    net = pvr.Net(batch_max=8, seed=4)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    dev = lambda a: torch.as_tensor(a, device="cuda")
    Y, S, V, T = dev(y), dev(s), dev(valid), dev(target)
    loss = torch.zeros(1, device="cuda")
    losses = []
    for _ in range(60):
        net.train_step(Y, S, V, pt, 0, B, T, 3e-3, loss)
        losses.append(float(loss))
    assert losses[-1] < 0.3 * losses[0], losses[::10]


def test_proposal_keeps_the_better_pose(pvr):
    """pvr_pose_propose: every output pose is the plain pose or the proposed
    one, and NCC at the output is never below NCC at the plain pose."""
    from paper_1611_07289_b300 import proposal, synth
    cfg = synth.config_tiny(noise=False)
    geom = cfg["geom"]
    desc, npix = synth.all_patches(geom, 64, 64)
    ctx = pvr.Context(geom, pvr.default_params(max_patches=256, max_pixels=1 << 20, max_patch_side=64))
    pt = pvr.PatchTable.from_numpy(desc, npix)
    x = torch.as_tensor(cfg["gt"], device="cuda")
    zeros = torch.zeros((pt.n, 6), dtype=torch.float64, device="cuda")
    y, _ = ctx.pvr_simulate(x, pt, zeros)
    rng = np.random.default_rng(5)
    poses = torch.as_tensor(synth.random_poses(rng, pt.n, rot=6.0, trans=3.0), device="cuda")
    net = pvr.Net(batch_max=16, seed=9)
    net.reserve(pt.n, npix)
    out = poses.clone()
    acc = torch.zeros(pt.n, dtype=torch.int32, device="cuda")
    net.propose(ctx, x, y, pt, out, proposal.SCALE, acc)
    n0, _ = ctx.pvr_ncc_grad(x, y, pt, poses, want_grad=False)
    n1, _ = ctx.pvr_ncc_grad(x, y, pt, out, want_grad=False)
    same = torch.all(out == poses, dim=1)
    assert torch.equal(same, acc == 0)
    assert torch.all(n1[~same] > n0[~same]) and torch.all(n1[same] == n0[same])
