"""Measured error of every GPU result against the FP64 oracle (FP32 kernels)
and of the BF16 network against its float32 reference.

Not a test: it prints one markdown table row per result (the largest error
over the cases listed, with the tolerance the parity tests hold it to).
Run on a GPU:  python tests/error_table.py
"""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import cnn_ref  # noqa: E402
from oracle import pvr_oracle as O  # noqa: E402
from paper_1611_07289_b300 import pvr, synth  # noqa: E402
from tests.cases import rel_l2, tiled_case, uneven_case  # noqa: E402

ROWS = []


def row(result, measure, value, tol, cases):
    ROWS.append((result, measure, value, tol, cases))


def t(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def ctx_for(geom, dz=0.8, **kw):
    return pvr.Context(geom, pvr.default_params(psf_dz=dz, max_patches=4096, max_pixels=1 << 22,
                                                max_patch_side=256, **kw))


def forward_and_adjoint():
    lat, sim_e, valid_mm, adj_a, adj_c = 0, 0.0, 0, 0.0, 0.0
    for case in (uneven_case, tiled_case):
        for n_params in (6, 12):
            geom, desc, npix, poses, rng = case()
            if n_params == 12:
                poses = np.concatenate([poses[:, :3], rng.uniform(-0.1, 0.1, (len(poses), 9))], 1)
            x = rng.uniform(0, 1000, geom.n_vox).astype(np.float32)
            r = rng.normal(size=npix).astype(np.float32)
            w = rng.uniform(0, 1, npix).astype(np.float32)
            ctx = ctx_for(geom, n_params=n_params)
            pt = pvr.PatchTable.from_numpy(desc, npix)
            G, ps = O.geom(geom), O.psf(1.2, 1, 3, 0.8)
            fix = O.pose_fixed(G, ps, desc, poses, n_params)
            gf = ctx.pvr_pose_to_fixed(pt, t(poses)).cpu().numpy()[:, :13].astype(np.int64)
            lat += int(np.sum(gf != fix[:, :13]))
            s, v = ctx.pvr_simulate(t(x), pt, t(poses))
            rs, rv, _ = O.simulate(G, ps, x, desc, fix, npix)
            valid_mm += int(np.sum(v.cpu().numpy() != rv))
            sim_e = max(sim_e, rel_l2(s.cpu().numpy(), rs))
            a, c = ctx.pvr_adjoint(pt, t(poses), t(r), t(w))
            ra, rc = O.adjoint(G, ps, desc, fix, r=r.astype(np.float64), w=w.astype(np.float64))
            adj_a = max(adj_a, rel_l2(a.cpu().numpy(), ra))
            adj_c = max(adj_c, rel_l2(c.cpu().numpy(), rc))
            ctx.close()
    cases = "uneven 1-33 px and multi-tile 3-130 px patches, rigid and affine poses"
    row("fixed-point lattice (a2)", "entries differing", lat, "0 (bit-exact)", cases)
    row("simulate valid mask (a3)", "pixels differing", valid_mm, "0 (bit-exact)", cases)
    row("simulate (a3)", "rel L2", sim_e, "1e-5", cases)
    row("adjoint addon = A^T(w r) (a6)", "rel L2", adj_a, "1e-5", cases)
    row("adjoint conf = A^T w (a6)", "rel L2", adj_c, "1e-5", cases)


def em_and_update():
    cfg = synth.config_tiny()
    geom = cfg["geom"]
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 1.0)
    desc, npix = O.patches_build(G, synth.pack_stacks(cfg["stacks"]), 32, 16)
    y = synth.pack_patch_pixels(cfg["stacks"], desc)
    poses = np.zeros((desc.shape[0], 6))
    fix = O.pose_fixed(G, ps, desc, poses)
    x = O.volume_init(G, ps, desc, fix, y).astype(np.float32)
    sim, valid, _ = O.simulate(G, ps, x, desc, fix, npix)
    ctx = ctx_for(geom, dz=1.0)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    st, sto = pvr.new_state(), O.new_state()
    mask = torch.ones(desc.shape[0], dtype=torch.uint8, device="cuda")
    mo = np.ones(desc.shape[0], np.uint8)
    e_p = e_s = e_c = e_pb = 0.0
    mm = 0
    for _ in range(3):
        p, wp, pb, m_out = ctx.pvr_em_weights(t(y), t(sim.astype(np.float32)), t(valid), pt, st, mask)
        rp, rwp, rpb, rmo = O.em_weights(y, sim.astype(np.float32).astype(np.float64), valid, desc,
                                         O.em_params(), sto, mo)
        sg = st.cpu().numpy()
        e_p = max(e_p, rel_l2(p.cpu().numpy(), rp))
        e_pb = max(e_pb, rel_l2(pb.cpu().numpy(), rpb))
        e_s = max(e_s, abs(sg[O.ST["SIGMA2"]] - sto[O.ST["SIGMA2"]]) / sto[O.ST["SIGMA2"]])
        e_c = max(e_c, abs(sg[O.ST["C"]] - sto[O.ST["C"]]) / sto[O.ST["C"]])
        near = np.abs(rwp - 0.5) < 1e-4
        mm += int(np.sum(m_out.cpu().numpy()[~near] != rmo[~near]))
        mask, mo = m_out.clone(), rmo
    cases = "64^3 workload, 540 patches, 3 warm-started calls"
    row("EM pixel weights p (a4)", "rel L2", e_p, "1e-5", cases)
    row("EM sigma^2 (a4/a5, float64 sums)", "rel", e_s, "1e-5", cases)
    row("EM inlier proportion c (a5)", "rel", e_c, "1e-5", cases)
    row("patch potentials p-bar (a5)", "rel L2", e_pb, "1e-5", cases)
    row("patch masks (a5)", "patches differing (away from w = 0.5 +- 1e-4)", mm, "0", cases)
    rng = np.random.default_rng(3)
    addon = rng.normal(0, 50, geom.n_vox).astype(np.float32)
    conf = np.abs(rng.normal(0, 1, geom.n_vox)).astype(np.float32)
    xg = t(x.copy())
    ctx.pvr_volume_update(xg, t(addon), t(conf), clear=False)
    xo = O.volume_update(x.astype(np.float64), addon.astype(np.float64), conf.astype(np.float64))
    row("SIRT update (a7)", "rel L2", rel_l2(xg.cpu().numpy(), xo), "1e-6", "64^3 volume, random addon / conf")
    ctx.close()


def ncc_and_registration():
    cfg = synth.config_tiny(noise=True)
    geom = cfg["geom"]
    x = cfg["gt"].reshape(-1).astype(np.float32)
    desc, _ = synth.all_patches(geom, 32, 16)
    rng = np.random.default_rng(0)
    d = desc[rng.choice(desc.shape[0], 60, replace=False)].copy()
    off = 0
    for r in d:
        r[6] = off
        off += int(r[4] * r[5])
    y = synth.pack_patch_pixels(cfg["stacks"], d)
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 1.0)
    for n_params in (6, 12):
        poses = synth.random_poses(rng, len(d), rot=3.0, trans=2.0)
        if n_params == 12:
            poses = np.concatenate([poses[:, :3], rng.uniform(-0.05, 0.05, (len(d), 9))], 1)
        ctx = ctx_for(geom, dz=1.0, n_params=n_params)
        pt = pvr.PatchTable.from_numpy(d, off)
        ncc, grad = ctx.pvr_ncc_grad(t(x), t(y), pt, t(poses))
        ncc, grad = ncc.cpu().numpy(), grad.cpu().numpy()
        en, eg = 0.0, 0.0
        for s in range(len(d)):
            rn, rg = O.ncc_grad(G, ps, x, y, d[s], poses[s], n_params=n_params)
            en = max(en, abs(ncc[s] - rn))
            if rn != 0.0:
                eg = max(eg, np.linalg.norm(grad[s] - rg) / np.linalg.norm(rg))
        kind = "rigid" if n_params == 6 else "affine"
        row(f"NCC ({kind}, a8)", "max abs", en, "2e-5", "64^3 workload, 60 noisy patches")
        row(f"NCC pose gradient ({kind}, a8)", "max rel (per patch)", eg, "2e-3", "64^3 workload, 60 noisy patches")
        r = rng.normal(size=off).astype(np.float32)
        g = ctx.pvr_pose_grad(t(x), t(r), pt, t(poses)).cpu().numpy()
        ev = 0.0
        for s in range(len(d)):
            _, rg = O.sim_pose_vjp(G, ps, x, r.astype(np.float64), d[s], poses[s], n_params=n_params)
            if np.linalg.norm(rg) > 0:
                ev = max(ev, np.linalg.norm(g[s] - rg) / np.linalg.norm(rg))
        row(f"pose VJP of the forward model ({kind}, NEXT-2)", "max rel (per patch)", ev, "2e-3",
            "64^3 workload, 60 patches, random r")
        ctx.close()


def iteration():
    cfg = synth.config_tiny()
    geom = cfg["geom"]
    G, ps = O.geom(geom), O.psf(1.2, 1, 3, 1.0)
    desc, npix = O.patches_build(G, synth.pack_stacks(cfg["stacks"]), 32, 16)
    y = synth.pack_patch_pixels(cfg["stacks"], desc)
    P = desc.shape[0]
    poses = np.zeros((P, 6))
    x0 = O.volume_init(G, ps, desc, O.pose_fixed(G, ps, desc, poses), y).astype(np.float32)
    ctx = ctx_for(geom, dz=1.0, reg_fixed_step=1, reg_delta0=0.25, reg_evals=3, n_sr=2)
    pt = pvr.PatchTable.from_numpy(desc, npix)
    xg, pg = t(x0.reshape(64, 64, 64)), t(poses)
    st = pvr.new_state()
    mask = torch.ones(P, dtype=torch.uint8, device="cuda")
    ctx.pvr_reconstruct_iter(xg, t(y), pt, pg, st, mask)
    xo, po, mo, _ = O.reconstruct_iter(G, ps, O.em_params(), O.reg_params(n_eval=3, fixed_step=1, delta0=0.25),
                                       x0, y, desc, poses, npix, O.new_state(), np.ones(P, np.uint8), n_sr=2)
    row("full outer iteration, fixed steps: volume", "rel L2", rel_l2(xg.cpu().numpy(), xo), "1e-4",
        "64^3 workload, 3 evaluations, 2 SR passes")
    row("full outer iteration, fixed steps: poses", "max abs (mm, degrees)", float(np.max(np.abs(pg.cpu().numpy() - po))),
        "1e-3", "same")
    ctx.close()
    # the benchmark's form: acceptance rule, forward model kept by the registration
    ctx = ctx_for(geom, dz=1.0, reg_evals=4, n_sr=1, reg_delta0=0.5)
    xg, pg = t(x0.reshape(64, 64, 64)), t(poses)
    st = pvr.new_state()
    mask = torch.ones(P, dtype=torch.uint8, device="cuda")
    ctx.pvr_reconstruct_iter(xg, t(y), pt, pg, st, mask)
    fix = O.pose_fixed(G, ps, desc, pg.cpu().numpy())
    xo, _ = O.sr_pass(G, ps, O.em_params(), x0, y, desc, fix, npix, O.new_state(), np.ones(P, np.uint8))
    row("iteration as benchmarked (accept iff NCC rises, kept forward model): SR at the GPU's poses",
        "rel L2", rel_l2(xg.cpu().numpy(), xo), "1e-4", "64^3 workload, 4 evaluations, 1 SR pass")
    ctx.close()


def cnn():
    rng = np.random.default_rng(0)
    B = 8
    desc = np.array([[0, 0, 0, 0, 64, 64, 4096 * b, 0] for b in range(B)], dtype=np.int32)
    npix = 4096 * B
    yy, xx = np.meshgrid(np.arange(64), np.arange(64), indexing="ij")
    y, s = np.zeros(npix, np.float32), np.zeros(npix, np.float32)
    for b in range(B):
        cx, cy, r = rng.uniform(16, 48), rng.uniform(16, 48), rng.uniform(6, 20)
        img = 300 + 500 * (((xx - cx) ** 2 + (yy - cy) ** 2) < r * r) + rng.normal(0, 20, (64, 64))
        y[4096 * b:4096 * (b + 1)] = img.reshape(-1)
        s[4096 * b:4096 * (b + 1)] = np.roll(img, tuple(rng.integers(-4, 5, 2)), axis=(0, 1)).reshape(-1)
    valid = np.ones(npix, np.uint8)
    target = rng.normal(0, 1, (B, 6)).astype(np.float32)
    net = pvr.Net(batch_max=B, seed=3)
    flat = net.get_params()
    pt = pvr.PatchTable.from_numpy(desc, npix)
    out = net.forward(t(y), t(s), t(valid), pt).cpu().numpy()
    loss = torch.zeros(1, device="cuda")
    net.train_step(t(y), t(s), t(valid), pt, 0, B, t(target), 1e-12, loss)
    g = net.get_grads()
    img = cnn_ref.inputs(y, s, valid, desc)
    for emulate, name in ((False, "float32 reference"), (True, "reference rounding to bf16 where the GPU stores bf16")):
        lr, orf, gr = cnn_ref.loss_and_grads(flat, img, target, emulate_bf16=emulate)
        row(f"CNN outputs (bf16 tcgen05, NEXT-3) vs {name}", "rel L2", rel_l2(out, orf), "1e-2", "8 synthetic pairs")
        row(f"CNN loss vs {name}", "rel", abs(float(loss) - lr) / lr, "1e-2", "same")
        row(f"CNN parameter gradient vs {name}", "rel L2 (all parameters)", rel_l2(g, gr), "3e-2 per layer", "same")


def main():
    torch.cuda.set_device(0)
    forward_and_adjoint()
    em_and_update()
    ncc_and_registration()
    iteration()
    cnn()
    print("| result | measure | measured error | test tolerance | cases |")
    print("|---|---|---|---|---|")
    for r, m, v, tol, cases in ROWS:
        vs = f"{v:.2e}" if isinstance(v, float) else str(v)
        print(f"| {r} | {m} | {vs} | {tol} | {cases} |")


if __name__ == "__main__":
    main()
