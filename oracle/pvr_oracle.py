"""Python wrapper of the FP64 CPU oracle (``oracle/pvr_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the product package never imports it
and shares no code with it.

Each function states the step of the PVR method (Alansary et al.,
arXiv:1611.07289) it follows; the C file carries the full definitions.
``reconstruct_iter`` strings the steps together in the paper's loop order
(Sec. II: register patches, then super-resolution with EM outlier weights).

Inputs are numpy arrays; geometry objects are duck-typed (attributes
``vol_dims``, ``w2v``, ``stack_dims``, ``p2w``, ``thickness``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pvr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libpvr_oracle.so")
_lock = threading.Lock()
_lib = None

MAX_STACKS = 16
ST = dict(INIT=0, SIGMA2=1, C=2, M=3, MU_P=4, SIGMA2_P=5, C_P=6, M_P=7, N_PART=8, SUM_P=9,
          SUM_PE2=10, EMIN=11, EMAX=12, N_ELIG=13, N_IN=14, SIGMA2_USED=15)


class _Geom(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("n_stacks", C.c_int),
                ("sw", C.c_int * MAX_STACKS), ("sh", C.c_int * MAX_STACKS),
                ("sk", C.c_int * MAX_STACKS), ("w2v", C.c_double * 12),
                ("p2w", (C.c_double * 12) * MAX_STACKS), ("thick", C.c_double * MAX_STACKS)]


class _Psf(C.Structure):
    _fields_ = [("fwhm_xy", C.c_double), ("kxy", C.c_int), ("kz", C.c_int), ("dz", C.c_double),
                ("kind", C.c_int), ("eps", C.c_double)]


class _EmParams(C.Structure):
    _fields_ = [("c0", C.c_double), ("sigma_floor_rel", C.c_double), ("min_valid_frac", C.c_double),
                ("patch_rule", C.c_int), ("patch_threshold", C.c_double),
                ("patch_em_iters", C.c_int)]


class _RegParams(C.Structure):
    _fields_ = [("n_params", C.c_int), ("n_eval", C.c_int), ("delta0", C.c_double),
                ("delta_min", C.c_double), ("fixed_step", C.c_int), ("min_valid", C.c_int),
                ("grow", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math, no FP contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or (
                os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
            os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fopenmp", "-ffp-contract=off",
                   "-fno-fast-math", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.POINTER
        L.or_pose_fixed_all.argtypes = [P(_Geom), P(_Psf), P(C.c_int), P(C.c_double), C.c_int,
                                        C.c_int, P(C.c_int64)]
        L.or_simulate.argtypes = [P(_Geom), P(_Psf), P(C.c_float), P(C.c_int), P(C.c_int64),
                                  C.c_int, P(C.c_double), P(C.c_uint8), P(C.c_double)]
        L.or_adjoint.argtypes = [P(_Geom), P(_Psf), P(C.c_int), P(C.c_int64), C.c_int,
                                 P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double)]
        L.or_em_weights.argtypes = [P(C.c_float), P(C.c_double), P(C.c_uint8), P(C.c_int), C.c_int,
                                    P(_EmParams), P(C.c_double), P(C.c_uint8), P(C.c_uint8),
                                    P(C.c_double), P(C.c_double), P(C.c_double)]
        L.or_sr_update.argtypes = [P(C.c_double), P(C.c_double), P(C.c_double), C.c_int, C.c_int, C.c_int,
                                   C.c_double, C.c_double, C.c_double, C.c_double]
        L.or_volume_update.argtypes = [P(C.c_double), P(C.c_double), P(C.c_double), C.c_size_t,
                                       C.c_double, C.c_double]
        L.or_ncc_grad.argtypes = [P(_Geom), P(_Psf), P(C.c_float), P(C.c_float), P(C.c_int),
                                  P(C.c_double), C.c_int, C.c_int, C.c_int, P(C.c_uint8), P(C.c_double)]
        L.or_ncc_grad.restype = C.c_double
        L.or_sim_pose_vjp.argtypes = [P(_Geom), P(_Psf), P(C.c_float), P(C.c_double), P(C.c_int),
                                      P(C.c_double), C.c_int, C.c_int, P(C.c_uint8), P(C.c_double)]
        L.or_sim_pose_vjp.restype = C.c_double
        L.or_register.argtypes = [P(_Geom), P(_Psf), P(_RegParams), P(C.c_float), P(C.c_float),
                                  P(C.c_int), C.c_int, P(C.c_double), P(C.c_double), P(C.c_double)]
        L.or_metrics.argtypes = [P(C.c_double), P(C.c_double), P(C.c_uint8), C.c_size_t,
                                 P(C.c_double)]
        L.or_patches_build.argtypes = [P(_Geom), P(C.c_float), C.c_int, C.c_int, C.c_double,
                                       C.c_double, P(C.c_int), C.c_int, P(C.c_int64)]
        L.or_patches_build.restype = C.c_int
        L.or_patches_build_sizes.argtypes = [P(_Geom), P(C.c_float), P(C.c_int), P(C.c_int),
                                             C.c_double, C.c_double, P(C.c_int), C.c_int,
                                             P(C.c_int64)]
        L.or_patches_build_sizes.restype = C.c_int
        L.or_patch_metrics.argtypes = [P(C.c_float), P(C.c_float), P(C.c_uint8), P(C.c_int), C.c_int,
                                       C.c_int, P(C.c_double), P(C.c_double)]
        L.or_psf_table.argtypes = [P(_Geom), P(_Psf), C.c_int, P(C.c_double), P(C.c_double)]
        _lib = L
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ctype))


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def geom(g) -> _Geom:
    """ctypes geometry from a geometry object."""
    G = _Geom()
    G.nx, G.ny, G.nz = (int(v) for v in g.vol_dims)
    G.n_stacks = len(g.stack_dims)
    assert G.n_stacks <= MAX_STACKS
    for r in range(12):
        G.w2v[r] = float(np.asarray(g.w2v, dtype=np.float64).reshape(12)[r])
    for s, (W, H, K) in enumerate(g.stack_dims):
        G.sw[s], G.sh[s], G.sk[s] = int(W), int(H), int(K)
        p = np.asarray(g.p2w[s], dtype=np.float64).reshape(12)
        for r in range(12):
            G.p2w[s][r] = float(p[r])
        G.thick[s] = float(g.thickness[s])
    return G


def psf(fwhm_xy=1.2, kxy=1, kz=3, dz=1.0, kind=0, eps=1e-12) -> _Psf:
    """kind 0: Gaussian in-plane PSF; kind 1: Taylor-series sinc in-plane."""
    return _Psf(float(fwhm_xy), int(kxy), int(kz), float(dz), int(kind), float(eps))


def em_params(c0=0.9, sigma_floor_rel=1e-3, min_valid_frac=0.1, patch_rule=0,
              patch_threshold=0.5, patch_em_iters=5) -> _EmParams:
    return _EmParams(c0, sigma_floor_rel, min_valid_frac, patch_rule, patch_threshold,
                     patch_em_iters)


def reg_params(n_params=6, n_eval=40, delta0=2.0, delta_min=0.01, fixed_step=0,
               min_valid=16, grow=1.0) -> _RegParams:
    return _RegParams(n_params, n_eval, delta0, delta_min, fixed_step, min_valid, grow)


def psf_table(G, ps, stack):
    gxy = np.zeros(33)
    gz = np.zeros(65)
    lib().or_psf_table(C.byref(G), C.byref(ps), int(stack), _ptr(gxy, C.c_double),
                       _ptr(gz, C.c_double))
    return gxy[:2 * ps.kxy + 1].copy(), gz[:2 * ps.kz + 1].copy()


def pose_fixed(G, ps, desc, poses, n_params=6):
    """Fixed-point sample lattice per patch (int64 [P, 16]); see or_pose_fixed."""
    desc = _c(desc, np.int32)
    poses = _c(poses, np.float64)
    P = desc.shape[0]
    fix = np.zeros((P, 16), dtype=np.int64)
    lib().or_pose_fixed_all(C.byref(G), C.byref(ps), _ptr(desc, C.c_int), _ptr(poses, C.c_double),
                            int(n_params), int(P), _ptr(fix, C.c_int64))
    return fix


def simulate(G, ps, x, desc, fix, npix):
    """Forward model (Eq. 1): returns sim (f64), valid (u8), den (f64)."""
    x = _c(x, np.float32)
    desc = _c(desc, np.int32)
    fix = _c(fix, np.int64)
    sim = np.zeros(npix, dtype=np.float64)
    valid = np.zeros(npix, dtype=np.uint8)
    den = np.zeros(npix, dtype=np.float64)
    lib().or_simulate(C.byref(G), C.byref(ps), _ptr(x, C.c_float), _ptr(desc, C.c_int),
                      _ptr(fix, C.c_int64), int(desc.shape[0]), _ptr(sim, C.c_double),
                      _ptr(valid, C.c_uint8), _ptr(den, C.c_double))
    return sim, valid, den


def adjoint(G, ps, desc, fix, r=None, w=None, nvox=None):
    """Transpose of simulate: returns (A^T (w r), A^T w) as f64 volumes."""
    desc = _c(desc, np.int32)
    fix = _c(fix, np.int64)
    if nvox is None:
        nvox = G.nx * G.ny * G.nz
    addon = np.zeros(nvox, dtype=np.float64)
    conf = np.zeros(nvox, dtype=np.float64)
    r = None if r is None else _c(r, np.float64)
    w = None if w is None else _c(w, np.float64)
    lib().or_adjoint(C.byref(G), C.byref(ps), _ptr(desc, C.c_int), _ptr(fix, C.c_int64),
                     int(desc.shape[0]), _ptr(r, C.c_double), _ptr(w, C.c_double),
                     _ptr(addon, C.c_double), _ptr(conf, C.c_double))
    return addon, conf


def new_state():
    return np.zeros(16, dtype=np.float64)


def em_weights(y, sim, valid, desc, ep, state, mask_in=None):
    """EM outlier weights (Eqs. m, p, p-bar).  state is updated in place.
    Returns p (f64), w_patch (f64), pbar (f64), mask_out (u8)."""
    y = _c(y, np.float32)
    sim = _c(sim, np.float64)
    valid = _c(valid, np.uint8)
    desc = _c(desc, np.int32)
    P = desc.shape[0]
    assert state.dtype == np.float64 and state.flags.c_contiguous
    mi = None if mask_in is None else _c(mask_in, np.uint8)
    mo = np.zeros(P, dtype=np.uint8)
    p = np.zeros(sim.shape[0], dtype=np.float64)
    wp = np.zeros(P, dtype=np.float64)
    pbar = np.zeros(P, dtype=np.float64)
    lib().or_em_weights(_ptr(y, C.c_float), _ptr(sim, C.c_double), _ptr(valid, C.c_uint8),
                        _ptr(desc, C.c_int), int(P), C.byref(ep), _ptr(state, C.c_double),
                        _ptr(mi, C.c_uint8), _ptr(mo, C.c_uint8), _ptr(p, C.c_double),
                        _ptr(wp, C.c_double), _ptr(pbar, C.c_double))
    return p, wp, pbar, mo


def volume_update(x, addon, conf, alpha=1.0, conf_eps=1e-6):
    """Weighted SIRT step; returns the new volume (f64)."""
    xo = np.array(x, dtype=np.float64, copy=True).reshape(-1)
    addon = _c(addon, np.float64).reshape(-1)
    conf = _c(conf, np.float64).reshape(-1)
    lib().or_volume_update(_ptr(xo, C.c_double), _ptr(addon, C.c_double), _ptr(conf, C.c_double),
                           xo.size, float(alpha), float(conf_eps))
    return xo


def sr_update(x, addon, conf, dims, alpha=1.0, conf_eps=1e-6, lam=0.0, delta=100.0):
    """SIRT step then the edge-preserving diffusion step (or_sr_update);
    dims = (nx, ny, nz); returns the new volume (f64, flat)."""
    xo = np.array(x, dtype=np.float64, copy=True).reshape(-1)
    addon = _c(addon, np.float64).reshape(-1)
    conf = _c(conf, np.float64).reshape(-1)
    nx, ny, nz = (int(v) for v in dims)
    lib().or_sr_update(_ptr(xo, C.c_double), _ptr(addon, C.c_double), _ptr(conf, C.c_double), nx, ny, nz,
                       float(alpha), float(conf_eps), float(lam), float(delta))
    return xo


def ncc_grad(G, ps, x, y, drow, theta, n_params=6, min_valid=16, exact=True, member=None):
    """NCC of one patch and its pose gradient; returns (ncc, grad).  member:
    uint8 per patch pixel (indexed like y) or None."""
    x = _c(x, np.float32)
    y = _c(y, np.float32)
    drow = _c(drow, np.int32)
    th = _c(theta, np.float64)
    m = None if member is None else _c(member, np.uint8)
    g = np.zeros(n_params, dtype=np.float64)
    v = lib().or_ncc_grad(C.byref(G), C.byref(ps), _ptr(x, C.c_float), _ptr(y, C.c_float),
                          _ptr(drow, C.c_int), _ptr(th, C.c_double), int(n_params), int(min_valid),
                          int(bool(exact)), _ptr(m, C.c_uint8), _ptr(g, C.c_double))
    return float(v), g


def sim_pose_vjp(G, ps, x, r, drow, theta, n_params=6, exact=True):
    """d (sum_pix r * sim) / d pose for one patch; returns (sum r * sim, grad).
    r is indexed like the patch pixels (offset drow[6])."""
    x = _c(x, np.float32)
    r = _c(r, np.float64)
    drow = _c(drow, np.int32)
    th = _c(theta, np.float64)
    g = np.zeros(n_params, dtype=np.float64)
    v = lib().or_sim_pose_vjp(C.byref(G), C.byref(ps), _ptr(x, C.c_float), _ptr(r, C.c_double),
                              _ptr(drow, C.c_int), _ptr(th, C.c_double), int(n_params),
                              int(bool(exact)), None, _ptr(g, C.c_double))
    return float(v), g


def register(G, ps, rp, x, y, desc, poses, margin=False):
    """Patch-wise gradient ascent on NCC; returns (new poses, best NCC per
    patch) and, with margin=True, also the smallest |NCC(trial) - NCC(best)|
    of each patch's acceptance decisions."""
    x = _c(x, np.float32)
    y = _c(y, np.float32)
    desc = _c(desc, np.int32)
    po = np.array(poses, dtype=np.float64, copy=True, order="C")
    ncc = np.zeros(desc.shape[0], dtype=np.float64)
    mg = np.zeros(desc.shape[0], dtype=np.float64)
    lib().or_register(C.byref(G), C.byref(ps), C.byref(rp), _ptr(x, C.c_float), _ptr(y, C.c_float),
                      _ptr(desc, C.c_int), int(desc.shape[0]), _ptr(po, C.c_double),
                      _ptr(ncc, C.c_double), _ptr(mg, C.c_double))
    return (po, ncc, mg) if margin else (po, ncc)


def metrics(ref, img, mask=None):
    """PSNR, CC, SSIM, DSSIM, MSE (Sec. IV-A)."""
    ref = _c(ref, np.float64).reshape(-1)
    img = _c(img, np.float64).reshape(-1)
    m = None if mask is None else _c(mask, np.uint8).reshape(-1)
    out = np.zeros(5, dtype=np.float64)
    lib().or_metrics(_ptr(ref, C.c_double), _ptr(img, C.c_double), _ptr(m, C.c_uint8), ref.size,
                     _ptr(out, C.c_double))
    return dict(psnr=out[0], cc=out[1], ssim=out[2], dssim=out[3], mse=out[4])


def patches_build(G, stacks, a, stride, fg_frac=0.0, keep_frac=0.0):
    """Square patch table (Sec. II "Patch Extraction"); returns (desc [P,8] int32, npix)."""
    stacks = _c(stacks, np.float32)
    npix = C.c_int64(0)
    n = lib().or_patches_build(C.byref(G), _ptr(stacks, C.c_float), int(a), int(stride),
                               float(fg_frac), float(keep_frac), None, 0, C.byref(npix))
    desc = np.zeros((max(n, 1), 8), dtype=np.int32)
    lib().or_patches_build(C.byref(G), _ptr(stacks, C.c_float), int(a), int(stride),
                           float(fg_frac), float(keep_frac), _ptr(desc, C.c_int), int(n),
                           C.byref(npix))
    return desc[:n], int(npix.value)


def volume_init(G, ps, desc, fix, y, conf_eps=1e-6):
    """Initial volume x0 = A^T y / A^T 1 at the initial poses (0 where unreached)."""
    addon, conf = adjoint(G, ps, desc, fix, r=np.asarray(y, dtype=np.float64), w=None)
    x = np.where(conf > conf_eps, addon / np.where(conf > conf_eps, conf, 1.0), 0.0)
    return x


def sr_pass(G, ps, ep, x, y, desc, fix, npix, state, mask_in, alpha=1.0, conf_eps=1e-6, lam=0.0, delta=100.0):
    """One super-resolution pass: simulate, EM weights, weighted adjoint of the
    residual, SIRT update (followed by the edge-preserving diffusion step
    when lam > 0).  Pixel weight = patch mask * p (an excluded patch
    contributes nothing).  Returns (x_new, aux dict)."""
    sim, valid, _ = simulate(G, ps, np.asarray(x, dtype=np.float32), desc, fix, npix)
    p, wp, pbar, mask = em_weights(y, sim, valid, desc, ep, state, mask_in)
    pix_mask = np.zeros(npix, dtype=np.float64)
    for s in range(desc.shape[0]):
        off, n = int(desc[s, 6]), int(desc[s, 4]) * int(desc[s, 5])
        pix_mask[off:off + n] = mask[s]
    e = np.where(valid > 0, np.asarray(y, dtype=np.float64) - sim, 0.0)
    wgt = pix_mask * p
    addon, conf = adjoint(G, ps, desc, fix, r=e, w=wgt)
    if lam > 0.0:
        xn = sr_update(np.asarray(x, dtype=np.float64), addon, conf, (G.nx, G.ny, G.nz), alpha, conf_eps, lam, delta)
    else:
        xn = volume_update(np.asarray(x, dtype=np.float64), addon, conf, alpha, conf_eps)
    return xn, dict(sim=sim, valid=valid, p=p, w_patch=wp, pbar=pbar, mask=mask, addon=addon,
                    conf=conf)


def reconstruct_iter(G, ps, ep, rp, x, y, desc, poses, npix, state, mask, n_sr=1, alpha=1.0,
                     conf_eps=1e-6, lam=0.0, delta=100.0):
    """One outer PVR iteration (Sec. II): register every patch to the current
    volume, then n_sr super-resolution passes with EM outlier weights.
    Returns (x, poses, mask, ncc)."""
    poses, ncc = register(G, ps, rp, np.asarray(x, dtype=np.float32), y, desc, poses)
    fix = pose_fixed(G, ps, desc, poses, rp.n_params)
    x = np.asarray(x, dtype=np.float64)
    for _ in range(n_sr):
        x, aux = sr_pass(G, ps, ep, x.astype(np.float32), y, desc, fix, npix, state, mask, alpha,
                         conf_eps, lam, delta)
        mask = aux["mask"]
    return x, poses, mask, ncc


def patches_build_sizes(G, stacks, slice_a, slice_stride, fg_frac=0.0, keep_frac=0.0):
    """Patch table with a side and stride per slice (slices over all stacks
    in order); returns (desc [P,8] int32, npix)."""
    stacks = _c(stacks, np.float32)
    sa = _c(slice_a, np.int32)
    ss = _c(slice_stride, np.int32)
    npix = C.c_int64(0)
    n = lib().or_patches_build_sizes(C.byref(G), _ptr(stacks, C.c_float), _ptr(sa, C.c_int),
                                     _ptr(ss, C.c_int), float(fg_frac), float(keep_frac), None, 0,
                                     C.byref(npix))
    desc = np.zeros((max(n, 1), 8), dtype=np.int32)
    lib().or_patches_build_sizes(C.byref(G), _ptr(stacks, C.c_float), _ptr(sa, C.c_int),
                                 _ptr(ss, C.c_int), float(fg_frac), float(keep_frac),
                                 _ptr(desc, C.c_int), n, C.byref(npix))
    return desc[:n], int(npix.value)


def patch_metrics(y, sim, valid, desc, w=3):
    """Per-patch {PSNR, CC, SSIM, DSSIM, mean local SSIM} (float64 [P, 5]) and
    the local DSSIM heat map (float64 [n_pix])."""
    y = _c(y, np.float32)
    sim = _c(sim, np.float32)
    valid = _c(valid, np.uint8)
    desc = _c(desc, np.int32)
    out = np.zeros((desc.shape[0], 5), dtype=np.float64)
    m = np.zeros(y.size, dtype=np.float64)
    lib().or_patch_metrics(_ptr(y, C.c_float), _ptr(sim, C.c_float), _ptr(valid, C.c_uint8),
                           _ptr(desc, C.c_int), int(desc.shape[0]), int(w), _ptr(out, C.c_double),
                           _ptr(m, C.c_double))
    return out, m
