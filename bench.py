"""Benchmark of the PVR hot path on the whole-uterus workload.

Workload (synthetic, seeded; the paper's fetal scans are not available):
256x256x192 volume at 0.75 mm, 4 stacks (3 orthogonal + 1 oblique 30 deg)
of 96 slices of 256x256 px at 0.75x0.75x2.5 mm, breathing + fetal motion,
5 % corrupted slices, square patches a = 64, stride 32, kept when half
their pixels exceed 1 % of the maximum.  Gaussian PSF kxy = 1, kz = 3,
dz = 0.75 mm.

One step = one pvr_reconstruct_iter: 2 NCC evaluations of every patch with
a registration accept/propose (affine poses, 12 parameters: the workload's
breathing motion is affine), the fixed-point lattice of the new poses,
simulate + residual, EM weights with patch classification, weighted adjoint,
SIRT update (every row of the hot-path table).  The patches are one tile
each, so the NCC kernels also leave the forward model and residual at each
patch's best pose, and the super-resolution pass takes them from there
instead of simulating a second time.  The patch table is built
once before timing.  value = patch-pixels processed per second (all ranks).

The line's "iteration" field times the method's whole outer iteration on the
same workload (registration until the step falls below 0.01 or 40 NCC
evaluations, then 5 super-resolution passes, each a SIRT step followed by
the edge-preserving diffusion step) for 10 outer iterations from the initial
volume, with the volume PSNR against the phantom after each: seconds per
iteration, the best and final PSNR, and the time to reach the best PSNR of
the same iterations without the regulariser ("iteration_unregularised",
where SIRT semi-converges: PSNR peaks after the first iteration and falls).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run; every rank runs an independent
replica of the workload (the method's cross-patch coupling is a volume
all-reduce that this single-GPU build does not implement), so scaling is
weak and value sums over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "patch-pixels/s for simulate+adjoint (and % HBM roofline); s/iteration at matched PSNR"
UNIT = "patch-pixels/s"
WORKLOAD = "pvr-uterus-256x256x192-4x96x256^2-a64s32"
L2_FLUSH_BYTES = 256 << 20


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _config_dict(n_patches=None, n_pix=None, slices=96):
    wl = WORKLOAD if slices == 96 else WORKLOAD.replace("4x96", f"4x{slices}")
    return {"workload": wl, "volume": [256, 256, 192], "voxel_mm": 0.75,
            "stacks": f"3 orthogonal + 1 oblique, {slices} x 256^2 @ 0.75x0.75x2.5 mm",
            "patch": 64, "stride": 32, "psf": "gaussian kxy=1 kz=3 dz=0.75mm",
            "step": "pvr_reconstruct_iter: 2 NCC evals + pose update, 1 SR pass",
            "pose": "affine, 12 parameters",
            "n_patches": n_patches, "n_patch_pixels": n_pix,
            "l2": "flushed between timed steps (256 MiB write)"}


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """SM clock and throttle reasons sampled every 20 ms during the timed
    region (NVML in a thread; nvidia-smi -lms 200 if NVML is unavailable)."""

    REASONS = {"hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
               "sw_power_cap": 0x4}

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.stop_flag = None
        self.thread = None
        self.proc = None
        self.path = None

    def start(self):
        try:
            import ctypes
            import threading
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")
            h = ctypes.c_void_p()
            if nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h)) != 0:
                raise OSError("no NVML handle")
            mx = ctypes.c_uint()
            nv.nvmlDeviceGetMaxClockInfo(h, ctypes.c_int(1), ctypes.byref(mx))   # 1 = SM clock
            self.max_mhz = mx.value
            reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
            self.stop_flag = threading.Event()

            def run():
                mhz, rs = ctypes.c_uint(), ctypes.c_ulonglong()
                while not self.stop_flag.is_set():
                    if nv.nvmlDeviceGetClockInfo(h, ctypes.c_int(1), ctypes.byref(mhz)) != 0:
                        break
                    if reasons_fn(h, ctypes.byref(rs)) != 0:
                        break
                    self.samples.append((mhz.value, rs.value))
                    self.stop_flag.wait(0.02)

            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            return
        except Exception as exc:  # no NVML: fall back to nvidia-smi sampling
            print(f"clock sampler: NVML unavailable ({exc!r}); using nvidia-smi", file=sys.stderr)
            self.thread = None
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", "--query-gpu=clocks.sm,clocks.max.sm,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.stop_flag.set()
            self.thread.join(timeout=2)
            if not self.samples:
                return None
            reasons = sorted({k for _, r in self.samples for k, bit in self.REASONS.items() if r & bit})
            return {"sm_mhz": statistics.median(m for m, _ in self.samples),
                    "sm_max_mhz": float(self.max_mhz), "reasons": reasons,
                    "samples": len(self.samples), "source": "nvml"}
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [[p.strip() for p in line.split(",")] for line in open(self.path)]
        rows = [r for r in rows if len(r) >= 6 and r[0].replace(".", "").isdigit()]
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(float(r[0]) for r in rows), "sm_max_mhz": float(rows[0][1]),
                "reasons": reasons, "samples": len(rows), "source": "nvidia-smi"}


# --------------------------------------------------------------- roofline --

def _algorithmic_bytes(cls, n_pix, n_vox):
    """Bytes a kernel class must move per launch group (each array read or
    written once; see the design notes for the per-unit figures)."""
    return {"simulate": 9 * n_pix + 4 * n_vox,        # y in, e out, valid out, x in
            "adjoint": 8 * n_pix + 8 * n_vox,         # e, p in; addon, conf out
            "em": 9 * n_pix,                          # e, valid in; p out
            # y in, x in (moments and gradient on chip), plus the kept forward
            # model: e and valid (5 B per pixel) written by the first of the
            # step's two evaluations -- 2.5 B per pixel per evaluation; the
            # second evaluation's rewrites for accepted trials are not counted
            "ncc": 4 * n_pix + 4 * n_vox + (5 * n_pix) // 2,
            "update": 24 * n_vox}.get(cls)            # x, addon, conf in; x, 0, 0 out


def _profile_traffic(cls):
    """Per-launch DRAM bytes of `cls` from the committed ncu summary, if the
    kernel source it was taken from is unchanged."""
    path = os.path.join(ROOT, "profiles", f"{cls}_uterus.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    if not m or not h:
        return None
    src = open(os.path.join(ROOT, "paper_1611_07289_b300", "csrc", "k_patch.cu"), "rb").read()
    if hashlib.sha256(src).hexdigest()[:16] != h.group(1)[:16]:
        return None
    return float(m.group(1))


_CLASS_KERNELS = {"ncc": ("k_ncc_fused", "k_ncc_moments"), "adjoint": ("k_adjoint",)}


def _profile_issue(cls):
    """Issue utilisation of the kernels of `cls` from the committed ncu
    counters (profiles/kernels_uterus24.md: smsp__issue_active, warp
    instructions, duration), if the kernel source is unchanged: the fraction
    of the SM schedulers' issue slots used while the kernel ran.  These
    kernels are gathers bound by instruction issue and load latency, so this
    is the bound that their HBM fraction does not show."""
    path = os.path.join(ROOT, "profiles", "kernels_uterus24.md")
    if cls not in _CLASS_KERNELS or not os.path.exists(path):
        return None
    txt = open(path).read()
    h = re.search(r"source_sha256 of csrc/k_patch.cu:\s*([0-9a-f]+)", txt)
    src = open(os.path.join(ROOT, "paper_1611_07289_b300", "csrc", "k_patch.cu"), "rb").read()
    if not h or hashlib.sha256(src).hexdigest()[:16] != h.group(1)[:16]:
        return None
    out = {}
    for k in _CLASS_KERNELS[cls]:
        m = re.search(r"## `" + k + r"`(.*?)(?=\n## |\Z)", txt, re.S)
        if not m:
            continue
        sec = m.group(1)
        ia = re.search(r"issue active % \(`smsp__issue_active[^`]*`\) \| ([0-9.]+)", sec)
        ls = re.search(r"stall long scoreboard / issue \([^)]*\) \| ([0-9.]+)", sec)
        bs = re.search(r"stall barrier / issue \([^)]*\) \| ([0-9.]+)", sec)
        if ia:
            out[k] = {"issue_active_frac": float(ia.group(1)) / 100.0,
                      "stall_long_scoreboard_per_issue": float(ls.group(1)) if ls else None,
                      "stall_barrier_per_issue": float(bs.group(1)) if bs else None}
    if not out:
        return None
    return {"bound": "issue", "kernels": out,
            "source": "ncu counters of the same kernel source, uterus geometry at 24 slices per stack "
                      "(profiles/kernels_uterus24.md)"}


L1_BYTES_PER_CLK_SM = 128   # nominal L1 load bandwidth of an SM


def _gathered_bytes(cls, desc, kxy=1, kz=3):
    """Trilinear corner bytes a gather kernel class reads per launch group:
    every lattice point of every patch (its w x h pixels plus a kxy halo)
    takes 2 kz + 1 through-plane samples of 8 float32 corners.  None for the
    scatter and streaming classes."""
    if cls not in ("simulate", "ncc"):
        return None
    w = desc[:, 4].astype(np.int64) + 2 * kxy
    h = desc[:, 5].astype(np.int64) + 2 * kxy
    return int((w * h).sum()) * (2 * kz + 1) * 8 * 4


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


# ----------------------------------------------------------- CPU (oracle) --

def _oracle_sample(cfg, desc_all, y_all, n_sample, seed=0):
    """A bounded sample of the workload for the FP64 oracle: n_sample patches
    drawn from the table (re-packed), with their acquired pixels."""
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(desc_all.shape[0], size=min(n_sample, desc_all.shape[0]), replace=False))
    d = desc_all[sel].copy()
    ys, off = [], 0
    for r in d:
        n = int(r[4] * r[5])
        ys.append(y_all[int(r[6]):int(r[6]) + n])
        r[6] = off
        off += n
    return d, np.concatenate(ys), off


N_PARAMS = 12   # affine patch poses (the workload's motion is affine)


def _oracle_step(O, G, ps, ep, rp, x, y, d, npix, state, mask):
    return O.reconstruct_iter(G, ps, ep, rp, x, y, d, np.zeros((d.shape[0], N_PARAMS)), npix, state, mask, n_sr=1)


def run_oracle(cfg, desc_all, y_all, budget_s=15.0, steps=1, warmup=0, log=print):
    """Time the oracle as it stands on a bounded sample; returns (rate, info)."""
    from oracle import pvr_oracle as O
    O.build()
    G, ps = O.geom(cfg["geom"]), O.psf(1.2, 1, 3, 0.75)
    ep, rp = O.em_params(), O.reg_params(n_params=N_PARAMS, n_eval=2)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    # size the sample: time 4 patches, scale to the budget
    d, y, npix = _oracle_sample(cfg, desc_all, y_all, 4)
    fix = O.pose_fixed(G, ps, d, np.zeros((d.shape[0], N_PARAMS)), N_PARAMS)
    x = O.volume_init(G, ps, d, fix, y).astype(np.float32)
    t0 = time.perf_counter()
    _oracle_step(O, G, ps, ep, rp, x, y, d, npix, O.new_state(), np.ones(d.shape[0], np.uint8))
    per_patch = max((time.perf_counter() - t0) / 4, 1e-4)
    n = int(max(4, min(desc_all.shape[0], budget_s / per_patch)))
    d, y, npix = _oracle_sample(cfg, desc_all, y_all, n, seed=1)
    fix = O.pose_fixed(G, ps, d, np.zeros((d.shape[0], N_PARAMS)), N_PARAMS)
    x = O.volume_init(G, ps, d, fix, y).astype(np.float32)
    for _ in range(warmup):
        _oracle_step(O, G, ps, ep, rp, x, y, d, npix, O.new_state(), np.ones(d.shape[0], np.uint8))
    times = []
    for _ in range(max(1, steps)):
        t0 = time.perf_counter()
        _oracle_step(O, G, ps, ep, rp, x, y, d, npix, O.new_state(), np.ones(d.shape[0], np.uint8))
        times.append(time.perf_counter() - t0)
    t = statistics.mean(times)
    info = {"kind": "oracle", "cores": cores, "sample": f"{d.shape[0]} of {desc_all.shape[0]} patches "
            f"({npix} patch-pixels), full volume, one reconstruct_iter (2 NCC evals + 1 SR pass, affine poses), "
            f"FP64 C oracle, OpenMP over patches", "step_s": t, "value": npix / t, "unit": UNIT}
    return npix / t, info


# ----------------------------------------------------------------- setup --

def _setup(device, slices=96, n_params=N_PARAMS, cfg=None):
    import torch
    from paper_1611_07289_b300 import pvr, synth
    t0 = time.perf_counter()
    if cfg is None:
        cfg = synth.config_uterus(device=device, slices=slices)
    gen_s = time.perf_counter() - t0
    packed = torch.as_tensor(synth.pack_stacks(cfg["stacks"]), device=device)
    prm = pvr.default_params(psf_dz=0.75, max_patches=32768, max_pixels=1 << 27, max_patch_side=64,
                             reg_evals=2, n_sr=1, n_params=n_params)
    ctx = pvr.Context(cfg["geom"], prm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pt, n = ctx.pvr_patches_build(packed, 64, 32, 0.01, 0.5)
    y = ctx.pvr_patches_gather(packed, pt)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    poses0 = torch.zeros((pt.n, n_params), dtype=torch.float64, device=device)
    x0 = ctx.pvr_volume_init(y, pt, poses0)
    torch.cuda.synchronize()
    return cfg, ctx, pt, y, x0, poses0, gen_s, build_s


SR_LAMBDA, SR_EDGE_DELTA = 0.5, 150.0   # regularised SR update of the whole-iteration field


def run_iterations(cfg, ctx_main, pt, y, x0, gt, dev, n_outer=10, reg_evals=40, n_sr=5, n_params=N_PARAMS,
                   lam=SR_LAMBDA, delta=SR_EDGE_DELTA, target=None, plan=None):
    """The method's whole outer iteration (registration to a step below 0.01
    or reg_evals evaluations, then n_sr SR passes, each a SIRT step followed
    -- lam > 0 -- by the edge-preserving diffusion step) repeated n_outer
    times from the initial volume; per-iteration device time (CUDA events)
    and the volume PSNR against the phantom after each; with `target`, the
    time at which PSNR first reaches it.  plan: (tile, mode) of the launch
    plan to make for the table (setup, untimed), which also fixes the
    spatial patch launch order."""
    import torch
    from paper_1611_07289_b300 import pvr
    prm = pvr.default_params(psf_dz=0.75, max_patches=32768, max_pixels=1 << 27, max_patch_side=64,
                             reg_evals=reg_evals, n_sr=n_sr, n_params=n_params, sr_lambda=lam,
                             sr_edge_delta=delta)
    ctx = pvr.Context(cfg["geom"], prm)
    if plan is not None:
        ctx.pvr_plan(pt, tile=plan[0], mode=plan[1])
    stream = torch.cuda.current_stream()
    x, poses = x0.clone(), torch.zeros((pt.n, n_params), dtype=torch.float64, device=dev)
    state, mask = pvr.new_state(dev), torch.ones(pt.n, dtype=torch.uint8, device=dev)
    psnr = [float(ctx.pvr_metrics(gt, x)[0])]
    ms = []
    l0 = ctx.launches
    for _ in range(n_outer):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.pvr_reconstruct_iter(x, y, pt, poses, state, mask)
        b.record(stream)
        psnr.append(float(ctx.pvr_metrics(gt, x)[0]))
        ms.append(a.elapsed_time(b))
    launches = ctx.launches - l0 - n_outer * 3   # the PSNR metric launches are not part of it
    ctx.pvr_device_status()
    ctx.close()
    best = int(np.argmax(psnr))
    cum = np.cumsum([0.0] + ms) * 1e-3
    reach = next((float(cum[i]) for i, v in enumerate(psnr) if target is not None and v >= target), None)
    sr = (f"SIRT step + edge-preserving diffusion (lambda {lam}, delta {delta})" if lam > 0
          else "SIRT step, no regulariser")
    return {"what": f"pvr_reconstruct_iter with reg_evals {reg_evals} (accept iff NCC rises, stop below step "
                    f"0.01), n_sr {n_sr} ({sr}), {'affine' if n_params == 12 else 'rigid'} poses, {n_outer} "
                    "outer iterations from the initial volume A^T y / A^T 1",
            "s_per_iteration": float(np.mean(ms)) * 1e-3, "ms_per_iteration": ms,
            "psnr_db": psnr, "best_psnr_db": psnr[best], "best_at_iteration": best,
            "s_to_best_psnr": float(cum[best]), "final_psnr_db": psnr[-1],
            "target_psnr_db": target, "s_to_target_psnr": reach,
            "gpu_launches_per_iteration": launches / n_outer,
            "stopping_rule": ("best PSNR (without the regulariser SIRT semi-converges and PSNR falls after it)"
                              if lam <= 0 else "PSNR rises at every iteration; the target is the unregularised "
                              "iteration's best PSNR")}


def run_ours(args, ws, rank, local, dist):
    import torch
    from paper_1611_07289_b300 import pvr
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    cfg, ctx, pt, y, x0, poses0, gen_s, build_s = _setup(dev, args.slices)
    n_pix, n_vox = pt.n_pix, cfg["geom"].n_vox
    # launch plan for simulate / adjoint tuned on this table (setup, untimed),
    # or the one given (profiling runs: the tuner's timings are distorted
    # under a profiler)
    if args.plan:
        tile, mode = (int(v) for v in args.plan.split(","))
        plan = ctx.pvr_plan(pt, x0, y, poses0, tile=tile, mode=mode)
    else:
        plan = ctx.pvr_plan(pt, x0, y, poses0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    gt = torch.as_tensor(cfg["gt"], device=dev)

    def fresh():
        return (x0.clone(), poses0.clone(), pvr.new_state(dev),
                torch.ones(pt.n, dtype=torch.uint8, device=dev))

    x, poses, state, mask = fresh()
    for _ in range(args.warmup):
        ctx.pvr_reconstruct_iter(x, y, pt, poses, state, mask)
    torch.cuda.synchronize()

    # device-timed region: inputs resident in HBM
    x, poses, state, mask = fresh()
    psnr0 = float(ctx.pvr_metrics(gt, x)[0])
    sampler = ClockSampler(local)
    launches0 = ctx.launches
    ctx.pvr_profile_enable(True)
    ctx.pvr_profile_read()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        ctx.pvr_reconstruct_iter(x, y, pt, poses, state, mask)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if dist:
        dist.barrier()
    prof = ctx.pvr_profile_read()
    ctx.pvr_profile_enable(False)
    launches = ctx.launches - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_ms = float(np.mean(step_ms))
    psnr1 = float(ctx.pvr_metrics(gt, x)[0])
    if dist:
        tt = torch.tensor([t_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())

    # end to end through the C ABI with host buffers: every step copies its
    # inputs (y, x, poses, EM state, mask) from pinned host memory and its
    # results (x, poses) back.  Steps are independent problems streamed
    # through the API: step k+1's upload and step k-1's download run on
    # copy streams while step k computes (two device buffer sets), so the
    # e2e time per step is the whole K-step region over K.  Each step's
    # inputs (~350 MB) exceed L2, so no flush is needed between steps.
    hy = y.cpu().pin_memory()
    hx, hp = x0.cpu().pin_memory(), poses0.cpu().pin_memory()
    hs = torch.zeros(16, dtype=torch.float64).pin_memory()
    hm = torch.ones(pt.n, dtype=torch.uint8).pin_memory()
    bufs = []
    for _ in range(2):
        bufs.append(dict(y=torch.empty_like(y), x=torch.empty_like(x0), p=torch.empty_like(poses0),
                         s=torch.empty(16, dtype=torch.float64, device=dev),
                         m=torch.empty(pt.n, dtype=torch.uint8, device=dev),
                         ox=torch.empty_like(hx).pin_memory(), op=torch.empty_like(hp).pin_memory(),
                         up=torch.cuda.Event(), done=torch.cuda.Event(), down=torch.cuda.Event()))
    h2d = hy.numel() * 4 + hx.numel() * 4 + hp.numel() * 8 + 16 * 8 + pt.n
    d2h = hx.numel() * 4 + hp.numel() * 8
    s_in, s_out, s_c = (torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev),
                        torch.cuda.Stream(device=dev))

    def e2e_run(n):
        for k in range(n):
            b = bufs[k % 2]
            with torch.cuda.stream(s_in):
                s_in.wait_event(b["down"])           # buffer set free (step k-2 downloaded)
                b["y"].copy_(hy, non_blocking=True)
                b["x"].copy_(hx, non_blocking=True)
                b["p"].copy_(hp, non_blocking=True)
                b["s"].copy_(hs, non_blocking=True)
                b["m"].copy_(hm, non_blocking=True)
                b["up"].record(s_in)
            s_c.wait_event(b["up"])
            ctx.pvr_reconstruct_iter(b["x"], b["y"], pt, b["p"], b["s"], b["m"], stream=s_c)
            b["done"].record(s_c)
            with torch.cuda.stream(s_out):
                s_out.wait_event(b["done"])
                b["ox"].copy_(b["x"], non_blocking=True)
                b["op"].copy_(b["p"], non_blocking=True)
                b["down"].record(s_out)

    for b in bufs:
        b["down"].record(s_out)
    e2e_run(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(s_in)
    e2e_run(args.steps)
    s_in.wait_stream(s_out)
    e1.record(s_in)
    torch.cuda.synchronize()
    e_t = e0.elapsed_time(e1) / args.steps
    if dist:
        tt = torch.tensor([e_t], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e_t = float(tt.item())

    if rank != 0:
        return None
    # roofline of the dominant kernel class
    peaks, peak_kind = _peaks()
    dom = max((k for k in prof if _algorithmic_bytes(k, 1, 1) is not None), key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / max(prof[dom][1], 1)
    abytes = _algorithmic_bytes(dom, n_pix, n_vox)
    achieved = abytes / (dom_ms * 1e-3) / 1e9
    traffic = _profile_traffic(dom)
    traffic_src = (f"dram__bytes_read.sum + dram__bytes_write.sum per launch from the committed ncu summary "
                   f"profiles/{dom}_uterus.md (cold-cache, serialised capture of the same kernel source)"
                   if traffic is not None else "no ncu capture of the current kernel source")
    breakdown = {k: {"ms_per_launch": v[0] / max(v[1], 1), "share": v[0] / max(sum(p[0] for p in prof.values()), 1e-12),
                     "launch_groups": v[1]} for k, v in prof.items() if v[1]}
    res = {
        "metric": METRIC, "value": ws * n_pix / (t_ms * 1e-3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(_config_dict(pt.n, n_pix, args.slices),
                       launch_plan={"tile": plan[0], "mode": ["one CTA per tile", "work queue"][plan[1]]}),
        "gpu_launches": int(launches),
        "e2e": {"value": ws * n_pix / (e_t * 1e-3), "unit": UNIT, "ms_per_step": e_t,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "traffic_source": traffic_src,
                     "algorithmic_bytes": abytes, "ms_per_launch": dom_ms,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                     else "fallback 6.4 TB/s"},
        "onchip": _onchip(dom, prof, pt, clocks),
        "issue": {c: _profile_issue(c) for c in ("ncc", "adjoint")},
        "kernels": breakdown,
        "clocks": clocks,
        "s_per_iteration": t_ms * 1e-3, "psnr_db": {"before": psnr0, "after_timed_steps": psnr1},
        "setup_s": {"generate": gen_s, "patch_table": build_s},
    }
    if not args.no_iteration:
        plain = run_iterations(cfg, ctx, pt, y, x0, gt, dev, n_outer=args.outer_full, lam=0.0, plan=plan[:2])
        res["iteration"] = run_iterations(cfg, ctx, pt, y, x0, gt, dev, n_outer=args.outer_full,
                                          target=plain["best_psnr_db"], plan=plan[:2])
        res["iteration_unregularised"] = plain
    if ws == 1 and not args.no_extras:
        # the batched uneven-patch form (NEXT-1) and the learned pose
        # proposal (NEXT-3) on the same volume and stacks, summarised
        ctx.close()
        u = run_uneven(args, ws, rank, local, cfg)
        res["batched_uneven"] = {k: u[k] for k in ("value", "unit", "ms_per_step", "simulate_adjoint_ms",
                                                   "iteration_ms", "roofline")}
        res["batched_uneven"]["config"] = u["config"]
        d = run_diff(args, ws, rank, local)
        res["differentiable"] = {k: d[k] for k in ("metric", "value", "unit", "ms_per_step",
                                                   "kernels_ms_per_step", "gpu_launches_per_step",
                                                   "descends", "config")}
        res["differentiable"]["loss_first_last"] = [d["loss"][0], d["loss"][-1]]
        res["differentiable"]["pose_error_first_last"] = [d["pose_mean_abs_error"][0],
                                                          d["pose_mean_abs_error"][-1]]
        p = run_proposal(args, ws, rank, local, cfg)
        res["learned_proposal"] = {k: p[k] for k in ("metric", "value", "unit", "plain_s_to_psnr",
                                                     "plain_best_psnr_db", "learned_best_psnr_db",
                                                     "s_to_psnr_per_run", "training", "config")}
    if ws == 1 and not args.no_cpu_baseline:
        _, info = run_oracle(cfg, pt.desc.cpu().numpy(), y.cpu().numpy(), budget_s=args.cpu_budget)
        res["cpu_baseline"] = {"value": info["value"], "unit": UNIT, "cores": info["cores"],
                               "kind": "oracle", "sample": info["sample"]}
    return res


def _onchip(dom, prof, pt, clocks):
    """The gather kernels' own bound: trilinear corner values read through L1
    per second against the nominal L1 load bandwidth at the SM clock seen."""
    import torch
    gb = _gathered_bytes(dom, pt.desc.cpu().numpy())
    if gb is None:
        return None
    ms = prof[dom][0] / max(prof[dom][1], 1)
    mhz = clocks.get("sm_mhz") or 2032.0
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    peak = n_sm * L1_BYTES_PER_CLK_SM * mhz * 1e6 / 1e9
    ach = gb / (ms * 1e-3) / 1e9
    return {"bound": "l1", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "gathered_bytes": gb, "what": "trilinear corner values gathered, 8 x 4 B per sample",
            "peak_source": f"nominal {L1_BYTES_PER_CLK_SM} B/clock/SM x {n_sm} SMs x {mhz:.0f} MHz"}


def run_uneven(args, ws, rank, local, cfg=None):
    """Batched patches of uneven sizes (sides 32..128 drawn per slice, stride
    side / 2) on the uterus volume: simulate + adjoint as one launch per
    patch size against one planned (tuned) launch over all sizes, and the
    whole iteration as direct calls against a captured CUDA graph."""
    import torch
    from paper_1611_07289_b300 import pvr, synth
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    t0 = time.perf_counter()
    cfg = synth.config_uneven(device=dev, slices=args.slices) if cfg is None else synth.uneven_sides(cfg)
    gen_s = time.perf_counter() - t0
    packed = torch.as_tensor(synth.pack_stacks(cfg["stacks"]), device=dev)
    prm = pvr.default_params(psf_dz=0.75, max_patches=65536, max_pixels=1 << 27, max_patch_side=128,
                             reg_evals=2, n_sr=1)
    ctx = pvr.Context(cfg["geom"], prm)
    pt, n = ctx.pvr_patches_build_sizes(packed, cfg["slice_a"], cfg["slice_stride"], 0.01, 0.5)
    y = ctx.pvr_patches_gather(packed, pt)
    poses0 = torch.zeros((pt.n, 6), dtype=torch.float64, device=dev)
    x0 = ctx.pvr_volume_init(y, pt, poses0)
    n_pix, n_vox = pt.n_pix, cfg["geom"].n_vox
    desc = pt.desc
    sides = sorted(set(desc[:, 4].tolist()))
    subs = []
    for a in sides:
        rows = torch.nonzero(desc[:, 4] == a).reshape(-1)
        subs.append((pvr.PatchTable(desc[rows].contiguous(), n_pix, a), poses0[rows].contiguous()))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    sim = torch.empty(n_pix, dtype=torch.float32, device=dev)
    valid = torch.empty(n_pix, dtype=torch.uint8, device=dev)
    addon = torch.empty_like(x0)
    conf = torch.empty_like(x0)

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return float(np.median(ms))

    def per_size():
        for k, (sub, ps) in enumerate(subs):
            ctx.pvr_simulate(x0, sub, ps, sim, valid)
            ctx.pvr_adjoint(sub, ps, y, None, addon, conf, accumulate=k > 0)

    def full():
        ctx.pvr_simulate(x0, pt, poses0, sim, valid)
        ctx.pvr_adjoint(pt, poses0, y, None, addon, conf)

    ctx.pvr_plan_clear()
    ms_size = timed(per_size, args.steps, args.warmup)
    ms_grid = timed(full, args.steps, args.warmup)
    plan = ctx.pvr_plan(pt, x0, y, poses0)
    ms_plan = timed(full, args.steps, args.warmup)

    x, poses = x0.clone(), poses0.clone()
    state, mask = pvr.new_state(dev), torch.ones(pt.n, dtype=torch.uint8, device=dev)

    def it_direct():
        ctx.pvr_reconstruct_iter(x, y, pt, poses, state, mask)

    ms_iter = timed(it_direct, args.steps, args.warmup)
    gs = torch.cuda.Stream(device=dev)
    x.copy_(x0)
    poses.copy_(poses0)
    state.zero_()
    mask.fill_(1)
    torch.cuda.synchronize()
    ctx.pvr_graph_capture(x, y, pt, poses, state, mask, stream=gs)
    gs.synchronize()
    sampler = ClockSampler(local)
    for _ in range(args.warmup):
        ctx.pvr_graph_launch(stream=gs)
    gs.synchronize()
    g_ms = []
    sampler.start()
    for _ in range(args.steps):
        with torch.cuda.stream(gs):
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(gs)
        ctx.pvr_graph_launch(stream=gs)
        b.record(gs)
        gs.synchronize()
        g_ms.append(a.elapsed_time(b))
    clocks = sampler.stop()
    ms_graph = float(np.median(g_ms))
    ctx.close()
    peaks, peak_kind = _peaks()
    abytes = _algorithmic_bytes("simulate", n_pix, n_vox) + _algorithmic_bytes("adjoint", n_pix, n_vox)
    achieved = abytes / (ms_plan * 1e-3) / 1e9
    counts = {int(a): int((desc[:, 4] == a).sum()) for a in sides}
    return {
        "metric": METRIC, "value": n_pix / (ms_graph * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "pvr-uterus-uneven-sides32-128-stride-half", "n_patches": pt.n,
                   "n_patch_pixels": n_pix, "patches_per_side": counts,
                   "step": "pvr_reconstruct_iter replayed from a captured CUDA graph",
                   "l2": "flushed between timed steps (256 MiB write)"},
        "simulate_adjoint_ms": {"one_launch_per_size": ms_size, "one_launch_grid": ms_grid,
                                "planned": ms_plan, "plan": {"tile": plan[0], "mode": plan[1],
                                                              "n_items": plan[2]}},
        "iteration_ms": {"direct_calls": ms_iter, "graph_replay": ms_graph},
        "roofline": {"bound": "hbm", "kernel": "simulate+adjoint (planned)", "achieved": achieved,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                     "traffic": None, "algorithmic_bytes": abytes, "ms_per_launch": ms_plan,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"},
        "clocks": clocks, "setup_s": {"generate": gen_s},
    }


def run_proposal(args, ws, rank, local, cfg=None):
    """Learned pose proposal on the uterus workload: train the CNN on pairs
    the forward model makes from random uterus phantoms, then reconstruct
    from the acquired positions with and without the proposal (+ NCC
    fallback) before registration, and compare PSNR against wall time."""
    import torch
    from paper_1611_07289_b300 import proposal, pvr
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    cfg, ctx, pt, y, x0, poses0, gen_s, build_s = _setup(dev, args.slices, n_params=6, cfg=cfg)
    gt = torch.as_tensor(cfg["gt"], device=dev)
    net = pvr.Net(batch_max=256, seed=7)
    net.reserve(pt.n, pt.n_pix)
    vols = proposal.phantom_volumes(cfg["geom"], range(100, 108), dev)
    losses, train_s = proposal.train(net, ctx, vols, pt, args.pairs, batch=256, lr=2e-3,
                                     log=lambda m: print(m, file=sys.stderr), geom=cfg["geom"])
    held = proposal.phantom_volumes(cfg["geom"], [200], dev)[0]
    before, after, taken = proposal.evaluate_proposal(net, ctx, held, pt, 2048, geom=cfg["geom"])

    def run(rctx, use_net):
        x, poses = x0.clone(), poses0.clone()
        state, mask = pvr.new_state(dev), torch.ones(pt.n, dtype=torch.uint8, device=dev)
        curve = [(0.0, float(rctx.pvr_metrics(gt, x)[0]))]
        t = 0.0
        for it in range(args.outer):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if use_net and it < args.propose_iters:
                net.propose(rctx, x, y, pt, poses, proposal.SCALE)
            rctx.pvr_reconstruct_iter(x, y, pt, poses, state, mask)
            torch.cuda.synchronize()
            t += time.perf_counter() - t0
            curve.append((t, float(rctx.pvr_metrics(gt, x)[0])))
        return curve

    # plain and learned registration at several evaluation budgets: the
    # proposal may let registration stop earlier, so each form is compared
    # at its own fastest setting
    curves = {}
    for evals in (2, 4, 10):
        prm = pvr.default_params(psf_dz=0.75, max_patches=32768, max_pixels=1 << 27, max_patch_side=64,
                                 reg_evals=evals, n_sr=2)
        rctx = pvr.Context(cfg["geom"], prm)
        rctx.pvr_plan(pt, x0, y, poses0)
        run(rctx, False)                      # warm-up of every kernel
        curves[f"plain_evals{evals}"] = run(rctx, False)
        curves[f"learned_evals{evals}"] = run(rctx, True)
        rctx.close()
    net.status()
    best_plain = max(p for k, c in curves.items() if k.startswith("plain") for _, p in c)
    target = best_plain - 0.1
    reach = {k: next((tt for tt, p in c if p >= target), None) for k, c in curves.items()}
    fastest = lambda kind: min((v for k, v in reach.items() if k.startswith(kind) and v is not None), default=None)
    return {
        "metric": "time to the plain method's best PSNR (within 0.1 dB), learned proposal vs plain",
        "value": fastest("learned"), "unit": "s", "higher_is_better": False, "n_gpus": 1,
        "plain_s_to_psnr": fastest("plain"), "plain_best_psnr_db": best_plain,
        "learned_best_psnr_db": max(p for k, c in curves.items() if k.startswith("learned") for _, p in c),
        "s_to_psnr_per_run": reach, "curves": curves,
        "training": {"pairs": args.pairs, "batch": 256, "seconds": train_s,
                     "loss_first_last": [losses[0], losses[-1]], "loss_predicting_zero": 2.0,
                     "phantoms": 8, "held_out_mean_abs_pose_error_before": before.tolist(),
                     "held_out_mean_abs_pose_error_after": after.tolist(), "held_out_taken_fraction": taken},
        "config": {"workload": WORKLOAD, "n_patches": pt.n, "outer_iterations": args.outer,
                   "reg_evals": [2, 4, 10], "n_sr": 2, "proposal_iterations": args.propose_iters,
                   "pose": "rigid (the network predicts rigid corrections)"},
        "data": "synthetic", "dtype": "bf16 network (tcgen05) / f32 reconstruction",
    }


def run_diff(args, ws, rank, local, steps=10, warmup=3):
    """Differentiable forward model: 128^3 nested-ellipsoid volume at 1 mm,
    3 orthogonal stacks of 86 slices of 128^2 at 1 x 1 x 1.5 mm, every 48 x 48
    patch at stride 24.  One step is one L2 gradient-descent step on the
    volume and the rigid poses through autograd.simulate_patches (forward
    pvr_simulate; backward pvr_adjoint for the volume, pvr_pose_grad for the
    poses) plus the loss and the update in torch; device-timed with CUDA
    events, L2 flushed between steps.  The data are simulated from the true
    volume at the true poses; the start is 0.8 x the volume and poses
    perturbed by up to 1 mm / 1 degree, so the loss and the pose error must
    fall at every step."""
    import torch
    from paper_1611_07289_b300 import pvr, synth
    from paper_1611_07289_b300.autograd import simulate_patches
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    cfg = synth.config_diff(device=dev)
    geom, desc, npix = cfg["geom"], cfg["desc"], cfg["n_pix"]
    ctx = pvr.Context(geom, pvr.default_params(psf_dz=1.0, max_patches=len(desc), max_pixels=npix,
                                               max_patch_side=48))
    pt = pvr.PatchTable.from_numpy(desc, npix, device=dev)
    x_true = torch.as_tensor(cfg["gt"].astype(np.float32), device=dev).reshape(ctx.vol_shape).contiguous()
    th_true = torch.zeros((pt.n, 6), dtype=torch.float64, device=dev)
    y, _ = ctx.pvr_simulate(x_true, pt, th_true)
    rng = np.random.default_rng(4)
    th0 = th_true + torch.as_tensor(synth.random_poses(rng, pt.n, rot=1.0, trans=1.0), device=dev)
    x0 = (x_true * 0.8).contiguous()
    plan = ctx.pvr_plan(pt, x0, y, th0)
    _, conf = ctx.pvr_adjoint(pt, th_true)
    ax = 1.0 / float(conf.max())      # below 2 / ||A^T A|| (rows of A sum to one)

    def step(x, th):
        sim, valid = simulate_patches(x, th, ctx, pt)
        r = (sim - y) * valid.float()
        loss = 0.5 * (r * r).sum()
        x.grad = th.grad = None
        loss.backward()
        with torch.no_grad():
            x -= ax * x.grad
            g = th.grad
            th -= 0.05 * g / g.norm(dim=1, keepdim=True).clamp_min(1e-30)
        return loss.detach()

    x, th = x0.clone().requires_grad_(True), th0.clone().requires_grad_(True)
    for _ in range(warmup):
        step(x, th)
    torch.cuda.synchronize()
    x, th = x0.clone().requires_grad_(True), th0.clone().requires_grad_(True)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    losses, perr = [], [(th.detach() - th_true).abs().mean()]
    l0 = ctx.launches
    ctx.pvr_profile_enable(True)
    ctx.pvr_profile_read()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        losses.append(step(x, th))
        ev[k][1].record(stream)
        perr.append((th.detach() - th_true).abs().mean())
    torch.cuda.synchronize()
    prof = ctx.pvr_profile_read()
    ctx.pvr_profile_enable(False)
    launches = ctx.launches - l0
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    losses = [float(v) for v in losses]
    perr = [float(v) for v in perr]
    ctx.pvr_device_status()
    ctx.close()
    return {
        "metric": "patch-pixels/s of one autograd step (forward model, volume and pose gradients, update)",
        "value": npix / (ms * 1e-3), "unit": "patch-pixels/s", "ms_per_step": ms, "steps": steps,
        "warmup": warmup,
        "kernels_ms_per_step": {k: v[0] / steps for k, v in prof.items() if v[1]},
        "gpu_launches_per_step": launches / steps,
        "loss": losses, "pose_mean_abs_error": perr,
        "descends": all(b < a for a, b in zip(losses, losses[1:])) and perr[-1] < perr[0],
        "config": {"workload": "diff-128: 128^3 at 1 mm, 3 x 86 slices of 128^2, 48x48 patches stride 24",
                   "n_patches": pt.n, "n_patch_pixels": npix, "pose": "rigid, 6 parameters",
                   "launch_plan": {"tile": plan[0], "mode": plan[1]},
                   "l2": "flushed between timed steps (256 MiB write)"},
        "data": "synthetic", "dtype": "f32",
    }


def _event_ms(fn, reps=5, warmup=2, flush=None):
    """Median device time (ms) of fn() over reps runs after warmup runs,
    CUDA events on the current stream, L2 flushed before each run."""
    import torch
    for _ in range(warmup):
        fn()
    ts = []
    s = torch.cuda.current_stream()
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def run_variants(args, ws, rank, local, cfg=None):
    """The paper's variants on the uterus workload, each timed through its
    library call (CUDA events, L2 flushed): the benchmark step with the
    Taylor-sinc in-plane PSF against the Gaussian one, the rigidity map, the
    per-patch metrics with local DSSIM maps, the superpixel patch table; and
    on the skew-motion workload (the paper's adult-brain motion model on a
    phantom) patches under rigid and affine poses and whole slices under
    rigid poses, PSNR after each outer iteration."""
    import torch
    from paper_1611_07289_b300 import pvr, synth
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    if cfg is None:
        cfg = synth.config_uterus(device=dev, slices=args.slices)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    packed = torch.as_tensor(synth.pack_stacks(cfg["stacks"]), device=dev)
    out = {}
    steps = {}
    for kind, name in ((0, "gaussian"), (1, "taylor_sinc")):
        prm = pvr.default_params(psf_dz=0.75, max_patches=32768, max_pixels=1 << 27, max_patch_side=64,
                                 reg_evals=2, n_sr=1, n_params=N_PARAMS, psf_kind=kind, slic_a_min=32)
        ctx = pvr.Context(cfg["geom"], prm)
        pt, n = ctx.pvr_patches_build(packed, 64, 32, 0.01, 0.5)
        y = ctx.pvr_patches_gather(packed, pt)
        P0 = torch.zeros((pt.n, N_PARAMS), dtype=torch.float64, device=dev)
        x0 = ctx.pvr_volume_init(y, pt, P0)
        ctx.pvr_plan(pt, x0, y, P0)
        x, P, st = x0.clone(), P0.clone(), pvr.new_state(dev)
        m = torch.ones(pt.n, dtype=torch.uint8, device=dev)
        steps[name] = _event_ms(lambda: ctx.pvr_reconstruct_iter(x, y, pt, P, st, m), flush=flush)
        if kind == 0:
            sim, valid = ctx.pvr_simulate(x0, pt, P0)
            st2 = pvr.new_state(dev)
            p, w, pbar, mk = ctx.pvr_em_weights(y, sim, valid, pt, st2)
            out["rigidity_map_ms"] = _event_ms(lambda: ctx.pvr_rigidity_map(pt, P0, p, pbar), flush=flush)
            out["patch_metrics_ms"] = _event_ms(lambda: ctx.pvr_patch_metrics(y, sim, valid, pt, w=3),
                                                flush=flush)
            res = {}

            def slic():
                res["t"] = ctx.pvr_patches_build_slic(packed, 32, 10.0, 2, n_iter=10)
            out["slic_patch_table_ms"] = _event_ms(slic, reps=3, warmup=1, flush=flush)
            spt, sn = res["t"]
            out["slic_patches"] = int(sn)
            out["slic_patch_pixels"] = int(spt.n_pix)
            out["n_patches"] = int(pt.n)
            out["n_patch_pixels"] = int(pt.n_pix)
        ctx.pvr_device_status()
        ctx.close()
    out["step_ms"] = steps
    # skew motion: patches under rigid (6) and affine (12) poses, and whole
    # slices under rigid poses (slice-to-volume registration), 4 outer
    # iterations with the regularised update
    sk = synth.config_skew(theta_deg=5.0, device=dev)
    gt = torch.as_tensor(sk["gt"], device=dev)
    spacked = torch.as_tensor(synth.pack_stacks(sk["stacks"]), device=dev)
    skew = {}
    for name, a, stride, npar in (("patches_rigid", 32, 16, 6), ("patches_affine", 32, 16, 12),
                                  ("slices_rigid", 96, 96, 6)):
        prm = pvr.default_params(psf_dz=sk["dz"], max_patches=32768, max_pixels=1 << 26, max_patch_side=96,
                                 reg_evals=20, n_sr=3, n_params=npar, sr_lambda=SR_LAMBDA,
                                 sr_edge_delta=SR_EDGE_DELTA)
        ctx = pvr.Context(sk["geom"], prm)
        pt, n = ctx.pvr_patches_build(spacked, a, stride, sk["fg_frac"], sk["keep_frac"] if a < 96 else 0.0)
        y = ctx.pvr_patches_gather(spacked, pt)
        P = torch.zeros((pt.n, npar), dtype=torch.float64, device=dev)
        x = ctx.pvr_volume_init(y, pt, P)
        ctx.pvr_plan(pt, tile=64, mode=0)
        st, m = pvr.new_state(dev), torch.ones(pt.n, dtype=torch.uint8, device=dev)
        psnr, ms = [float(ctx.pvr_metrics(gt, x)[0])], []
        for _ in range(4):
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record()
            ctx.pvr_reconstruct_iter(x, y, pt, P, st, m)
            b_.record()
            torch.cuda.synchronize()
            ms.append(a_.elapsed_time(b_))
            psnr.append(float(ctx.pvr_metrics(gt, x)[0]))
        skew[name] = {"n_patches": int(pt.n), "psnr_db": psnr, "ms_per_iteration": ms}
        ctx.pvr_device_status()
        ctx.close()
    skew["config"] = {"workload": "skew-5deg: 96^3 nested ellipsoids at 1.25 mm, 3 orthogonal stacks of 48 "
                                  "slices of 96^2, odd slices skewed (tan 5 deg); patches 32x32 stride 16 or "
                                  "whole slices",
                      "reg_evals": 20, "n_sr": 3, "outer_iterations": 4,
                      "sr_update": f"SIRT + diffusion (lambda {SR_LAMBDA}, delta {SR_EDGE_DELTA})"}
    out["skew_motion"] = skew
    out["config"] = {"workload": WORKLOAD, "step": "pvr_reconstruct_iter: 2 NCC evals + pose update, 1 SR pass",
                     "slic": "a = 32, compactness 10, dilation 2 px, 10 iterations (boxes above 64 px dropped)",
                     "l2": "flushed before each timed call (256 MiB write)"}
    out["data"] = "synthetic"
    return out


def run_reference(args, ws, rank):
    """The FP64 oracle as the reference arm: rank 0 only, on the host cores."""
    if rank != 0:
        return None
    import torch
    from paper_1611_07289_b300 import synth
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    cfg = synth.config_uterus(device=dev, slices=args.slices)
    from oracle import pvr_oracle as O
    O.build()
    desc, npix = O.patches_build(O.geom(cfg["geom"]), synth.pack_stacks(cfg["stacks"]), 64, 32, 0.01, 0.5)
    y = synth.pack_patch_pixels(cfg["stacks"], desc)
    # each step a bounded sample, so that K + W steps take about two minutes
    budget = min(args.cpu_budget, 120.0 / max(1, args.steps + args.warmup))
    rate, info = run_oracle(cfg, desc, y, budget_s=budget, steps=args.steps, warmup=args.warmup)
    return {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": info["step_s"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config_dict(int(desc.shape[0]), int(npix), args.slices),
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"]},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-iteration", action="store_true", help="skip the whole-iteration field")
    ap.add_argument("--plan", default="", help="force the simulate / adjoint launch plan: 'tile,mode' "
                    "(tile 32 or 64; mode 0 = one CTA per tile, 1 = work queue) instead of tuning it")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched uneven-patch, differentiable and learned-proposal fields")
    ap.add_argument("--outer-full", type=int, default=10, help="outer iterations of the whole-iteration field")
    ap.add_argument("--slices", type=int, default=96,
                    help="slices per stack (96 = the benchmark workload; fewer for profiling)")
    ap.add_argument("--workload", choices=["uterus", "uneven", "proposal", "diff", "variants"],
                    default="uterus",
                    help="uneven: patch sides 32..128 per slice (batched-launch comparison, 1 GPU); "
                         "proposal: learned pose proposal, time to PSNR against plain registration; "
                         "diff: autograd step of the differentiable forward model (128^3); "
                         "variants: the paper's variants (Taylor-sinc PSF, rigidity map, metrics, "
                         "superpixels, skew motion)")
    ap.add_argument("--pairs", type=int, default=200000, help="training pairs (proposal workload)")
    ap.add_argument("--outer", type=int, default=8, help="outer iterations (proposal workload)")
    ap.add_argument("--propose-iters", type=int, default=2, help="iterations that start with the proposal")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    ws, rank, local = _dist()
    dist = None
    if args.impl == "reference":
        res = run_reference(args, ws, rank)
    elif args.workload == "uneven":
        res = run_uneven(args, ws, rank, local) if rank == 0 else None
    elif args.workload == "proposal":
        res = run_proposal(args, ws, rank, local) if rank == 0 else None
    elif args.workload == "variants":
        res = run_variants(args, ws, rank, local) if rank == 0 else None
    elif args.workload == "diff":
        res = run_diff(args, ws, rank, local, steps=args.steps, warmup=args.warmup) if rank == 0 else None
    else:
        if ws > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl")
        res = run_ours(args, ws, rank, local, dist)
        if dist:
            dist.destroy_process_group()
    if res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
