"""Python binding of libpvr (the C ABI in include/pvr.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
Tensors are torch CUDA tensors (torch provides device memory and streams);
calls are enqueued on the current torch CUDA stream.  The library must have
been built (``python -m paper_1611_07289_b300.build``); importing this module
fails loudly if it is missing or cannot be loaded -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpvr.so")

MAX_STACKS = 16
EM_STATE_LEN = 16
ST = dict(INIT=0, SIGMA2=1, C=2, M=3, MU_P=4, SIGMA2_P=5, C_P=6, M_P=7, N_PART=8, SUM_P=9,
          SUM_PE2=10, EMIN=11, EMAX=12, N_ELIG=13, N_IN=14, SIGMA2_USED=15)
STATUS = {0: "PVR_OK", -1: "PVR_ERR_INVALID_ARG", -2: "PVR_ERR_CUDA", -3: "PVR_ERR_NUMERIC",
          -4: "PVR_ERR_BOUNDS", -5: "PVR_ERR_TIMEOUT", -6: "PVR_ERR_UNSUPPORTED"}


class PvrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Geometry(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("n_stacks", C.c_int32),
                ("stack_w", C.c_int32 * MAX_STACKS), ("stack_h", C.c_int32 * MAX_STACKS),
                ("stack_k", C.c_int32 * MAX_STACKS), ("world_to_voxel", C.c_double * 12),
                ("pixel_to_world", (C.c_double * 12) * MAX_STACKS),
                ("thickness", C.c_double * MAX_STACKS)]


class Params(C.Structure):
    _fields_ = [("psf_fwhm_xy", C.c_double), ("psf_kxy", C.c_int32), ("psf_kz", C.c_int32),
                ("psf_dz", C.c_double), ("alpha", C.c_double), ("conf_eps", C.c_double),
                ("em_c0", C.c_double), ("em_sigma_floor_rel", C.c_double),
                ("em_min_valid_frac", C.c_double), ("patch_rule", C.c_int32),
                ("patch_threshold", C.c_double), ("patch_em_iters", C.c_int32),
                ("n_params", C.c_int32), ("reg_evals", C.c_int32), ("reg_delta0", C.c_double),
                ("reg_delta_min", C.c_double), ("reg_grow", C.c_double),
                ("reg_fixed_step", C.c_int32), ("reg_min_valid", C.c_int32), ("n_sr", C.c_int32),
                ("max_patches", C.c_int32), ("max_pixels", C.c_int64),
                ("max_patch_side", C.c_int32), ("psf_kind", C.c_int32), ("psf_sinc_eps", C.c_double),
                ("slic_a_min", C.c_int32), ("sr_lambda", C.c_double), ("sr_edge_delta", C.c_double)]


class Patches(C.Structure):
    _fields_ = [("desc", C.c_void_p), ("n", C.c_int32), ("max_side", C.c_int32),
                ("n_pix", C.c_int64), ("member", C.c_void_p)]


_VP = C.c_void_p
_SIGS = {
    "pvr_params_default": (None, [C.POINTER(Params)]),
    "pvr_ctx_create": (C.c_int, [C.POINTER(_VP), C.POINTER(Geometry), C.POINTER(Params)]),
    "pvr_ctx_destroy": (C.c_int, [_VP]),
    "pvr_last_error": (C.c_char_p, [_VP]),
    "pvr_device_status": (C.c_int, [_VP, _VP]),
    "pvr_launch_count": (C.c_int64, [_VP]),
    "pvr_patches_build": (C.c_int, [_VP, _VP, C.c_int32, C.c_int32, C.c_double, C.c_double, _VP,
                                    C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int64), _VP]),
    "pvr_patches_build_sizes": (C.c_int, [_VP, _VP, _VP, _VP, C.c_double, C.c_double, _VP, C.c_int32,
                                          C.POINTER(C.c_int32), C.POINTER(C.c_int64), _VP]),
    "pvr_patches_build_slic": (C.c_int, [_VP, _VP, C.c_int32, C.c_double, C.c_int32, C.c_int32, C.c_double,
                                         C.c_double, _VP, _VP, C.c_int32, C.POINTER(C.c_int32),
                                         C.POINTER(C.c_int64), _VP]),
    "pvr_patches_gather": (C.c_int, [_VP, _VP, C.POINTER(Patches), _VP, _VP]),
    "pvr_pose_to_fixed": (C.c_int, [_VP, C.POINTER(Patches), _VP, _VP, _VP]),
    "pvr_simulate": (C.c_int, [_VP, _VP, C.POINTER(Patches), _VP, _VP, _VP, _VP]),
    "pvr_adjoint": (C.c_int, [_VP, C.POINTER(Patches), _VP, _VP, _VP, _VP, _VP, C.c_int32, _VP]),
    "pvr_em_weights": (C.c_int, [_VP, _VP, _VP, _VP, C.POINTER(Patches), _VP, _VP, _VP, _VP, _VP,
                                 _VP, _VP]),
    "pvr_volume_update": (C.c_int, [_VP, _VP, _VP, _VP, C.c_int32, _VP]),
    "pvr_volume_init": (C.c_int, [_VP, _VP, _VP, C.POINTER(Patches), _VP, _VP]),
    "pvr_ncc_grad": (C.c_int, [_VP, _VP, _VP, C.POINTER(Patches), _VP, _VP, _VP, _VP]),
    "pvr_pose_grad": (C.c_int, [_VP, _VP, _VP, C.POINTER(Patches), _VP, _VP, _VP]),
    "pvr_rigidity_map": (C.c_int, [_VP, C.POINTER(Patches), _VP, _VP, _VP, _VP, _VP]),
    "pvr_net_create": (C.c_int, [C.POINTER(_VP), C.c_int32, C.c_uint64]),
    "pvr_net_destroy": (C.c_int, [_VP]),
    "pvr_net_param_count": (C.c_int64, [_VP]),
    "pvr_net_get_params": (C.c_int, [_VP, _VP]),
    "pvr_net_set_params": (C.c_int, [_VP, _VP]),
    "pvr_net_get_grads": (C.c_int, [_VP, _VP]),
    "pvr_net_forward": (C.c_int, [_VP, _VP, _VP, _VP, C.POINTER(Patches), C.c_int32, C.c_int32, _VP, _VP]),
    "pvr_net_train_step": (C.c_int, [_VP, _VP, _VP, _VP, C.POINTER(Patches), C.c_int32, C.c_int32, _VP,
                                     C.c_float, _VP, _VP]),
    "pvr_net_reserve": (C.c_int, [_VP, C.c_int32, C.c_int64]),
    "pvr_net_status": (C.c_int, [_VP, _VP]),
    "pvr_pose_propose": (C.c_int, [_VP, _VP, _VP, _VP, C.POINTER(Patches), _VP, _VP, _VP, _VP]),
    "pvr_patch_metrics": (C.c_int, [_VP, _VP, _VP, _VP, C.POINTER(Patches), C.c_int32, _VP, _VP, _VP]),
    "pvr_plan": (C.c_int, [_VP, C.POINTER(Patches), _VP, _VP, _VP, C.c_int32, C.c_int32, _VP]),
    "pvr_plan_info": (C.c_int, [_VP, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "pvr_plan_clear": (C.c_int, [_VP]),
    "pvr_plan_order": (C.c_int, [_VP, _VP, C.c_int32, _VP]),
    "pvr_graph_capture": (C.c_int, [_VP, _VP, _VP, C.POINTER(Patches), _VP, _VP, _VP, _VP, _VP, _VP]),
    "pvr_graph_launch": (C.c_int, [_VP, _VP]),
    "pvr_register": (C.c_int, [_VP, _VP, _VP, C.POINTER(Patches), _VP, C.c_int32, _VP, _VP]),
    "pvr_reconstruct_iter": (C.c_int, [_VP, _VP, _VP, C.POINTER(Patches), _VP, _VP, _VP, _VP, _VP,
                                       _VP]),
    "pvr_metrics": (C.c_int, [_VP, _VP, _VP, _VP, C.c_int64, _VP, _VP]),
    "pvr_simulate_noalloc": (C.c_int, [C.POINTER(Geometry), C.POINTER(Params), _VP,
                                       C.POINTER(Patches), _VP, _VP, _VP, _VP]),
    "pvr_noalloc_status": (C.c_int, [_VP]),
    "pvr_profile_enable": (C.c_int, [_VP, C.c_int32]),
    "pvr_profile_read": (C.c_int, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_int64), _VP]),
}
KERNEL_CLASSES = ["pose", "simulate", "em", "adjoint", "update", "ncc", "ncc_finish", "reg_step"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpvr.so not built ({LIB_PATH}); run python -m paper_1611_07289_b300.build")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def exported_symbols():
    return sorted(_SIGS)


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def default_params(**kw) -> Params:
    p = Params()
    lib.pvr_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def geometry(g) -> Geometry:
    """ctypes geometry from a geometry object (vol_dims, w2v, stack_dims,
    p2w, thickness)."""
    G = Geometry()
    G.nx, G.ny, G.nz = (int(v) for v in g.vol_dims)
    G.n_stacks = len(g.stack_dims)
    w2v = np.asarray(g.w2v, dtype=np.float64).reshape(12)
    for i in range(12):
        G.world_to_voxel[i] = float(w2v[i])
    for s, (W, H, K) in enumerate(g.stack_dims):
        G.stack_w[s], G.stack_h[s], G.stack_k[s] = int(W), int(H), int(K)
        p = np.asarray(g.p2w[s], dtype=np.float64).reshape(12)
        for i in range(12):
            G.pixel_to_world[s][i] = float(p[i])
        G.thickness[s] = float(g.thickness[s])
    return G


class PatchTable:
    """Device patch table int32 [n, 8] plus the host-side counts the C ABI
    needs (pvr_patches)."""

    def __init__(self, desc: torch.Tensor, n_pix: int, max_side: int = 0, member=None):
        assert desc.dtype == torch.int32 and desc.is_cuda and desc.dim() == 2 and desc.shape[1] == 8
        self.desc = desc.contiguous()
        self.n = int(desc.shape[0])
        self.n_pix = int(n_pix)
        if max_side <= 0 and self.n > 0:
            max_side = int(desc[:, 4:6].max().item())
        self.max_side = int(max_side)
        self.member = None
        if member is not None:
            assert member.dtype == torch.uint8 and member.is_cuda and member.numel() >= self.n_pix
            self.member = member.contiguous()
        self.c = Patches(C.c_void_p(self.desc.data_ptr()) if self.n else None, self.n,
                         self.max_side, self.n_pix,
                         C.c_void_p(self.member.data_ptr()) if self.member is not None else None)

    @classmethod
    def from_numpy(cls, desc_np, n_pix, device="cuda"):
        d = torch.as_tensor(np.ascontiguousarray(desc_np, dtype=np.int32), device=device)
        ms = int(np.max(desc_np[:, 4:6])) if len(desc_np) else 0
        return cls(d, n_pix, ms)


class Context:
    """pvr_ctx: geometry, parameters and all scratch of the library."""

    def __init__(self, geom, params: Params | None = None, **kw):
        self.params = params if params is not None else default_params(**kw)
        self.geom_c = geometry(geom) if not isinstance(geom, Geometry) else geom
        self.vol_shape = (self.geom_c.nz, self.geom_c.ny, self.geom_c.nx)
        h = C.c_void_p()
        rc = lib.pvr_ctx_create(C.byref(h), C.byref(self.geom_c), C.byref(self.params))
        if rc != 0:
            raise PvrError(rc, "pvr_ctx_create failed (see stderr)")
        self.h = h
        self.n_params = int(self.params.n_params)

    def close(self):
        if getattr(self, "h", None):
            lib.pvr_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc):
        if rc != 0:
            raise PvrError(rc, lib.pvr_last_error(self.h).decode())

    @property
    def launches(self) -> int:
        return int(lib.pvr_launch_count(self.h))

    def pvr_device_status(self, stream=None):
        self._chk(lib.pvr_device_status(self.h, _stream(stream)))

    def pvr_patches_build(self, stacks, a, stride, fg_frac=0.0, keep_frac=0.0, max_out=None,
                          stream=None):
        if max_out is None:
            max_out = self.params.max_patches
        desc = torch.zeros((max(max_out, 1), 8), dtype=torch.int32, device=stacks.device)
        n = C.c_int32(0)
        npix = C.c_int64(0)
        self._chk(lib.pvr_patches_build(self.h, _ptr(stacks), int(a), int(stride), float(fg_frac),
                                        float(keep_frac), _ptr(desc), int(max_out), C.byref(n),
                                        C.byref(npix), _stream(stream)))
        nn = min(int(n.value), int(max_out))
        return PatchTable(desc[:nn].clone(), int(npix.value), int(a)), int(n.value)

    def pvr_patches_build_sizes(self, stacks, slice_a, slice_stride, fg_frac=0.0, keep_frac=0.0,
                                max_out=None, stream=None):
        """Patch table with a side and stride per slice (host int arrays, one
        entry per slice of every stack in order)."""
        if max_out is None:
            max_out = self.params.max_patches
        sa = np.ascontiguousarray(slice_a, dtype=np.int32)
        ss = np.ascontiguousarray(slice_stride, dtype=np.int32)
        desc = torch.zeros((max(max_out, 1), 8), dtype=torch.int32, device=stacks.device)
        n = C.c_int32(0)
        npix = C.c_int64(0)
        self._chk(lib.pvr_patches_build_sizes(self.h, _ptr(stacks), sa.ctypes.data, ss.ctypes.data,
                                              float(fg_frac), float(keep_frac), _ptr(desc), int(max_out),
                                              C.byref(n), C.byref(npix), _stream(stream)))
        nn = min(int(n.value), int(max_out))
        ms = int(sa.max()) if sa.size else 0
        return PatchTable(desc[:nn].clone(), int(npix.value), ms), int(n.value)

    def pvr_patches_build_slic(self, stacks, a, compactness, gamma, n_iter=10, fg_frac=0.0, keep_frac=0.0,
                               max_out=None, stream=None):
        """Superpixel patch table with membership masks (PatchTable.member)."""
        if max_out is None:
            max_out = self.params.max_patches
        desc = torch.zeros((max(max_out, 1), 8), dtype=torch.int32, device=stacks.device)
        member = torch.zeros(int(self.params.max_pixels), dtype=torch.uint8, device=stacks.device)
        n = C.c_int32(0)
        npix = C.c_int64(0)
        self._chk(lib.pvr_patches_build_slic(self.h, _ptr(stacks), int(a), float(compactness), int(gamma),
                                             int(n_iter), float(fg_frac), float(keep_frac), _ptr(desc),
                                             _ptr(member), int(max_out), C.byref(n), C.byref(npix),
                                             _stream(stream)))
        nn = min(int(n.value), int(max_out))
        d = desc[:nn].clone()
        ms = int(d[:, 4:6].max().item()) if nn else 1
        return PatchTable(d, int(npix.value), ms, member[:max(int(npix.value), 1)].clone()), int(n.value)

    def pvr_patches_gather(self, stacks, pt: PatchTable, y=None, stream=None):
        if y is None:
            y = torch.empty(pt.n_pix, dtype=torch.float32, device=stacks.device)
        self._chk(lib.pvr_patches_gather(self.h, _ptr(stacks), C.byref(pt.c), _ptr(y), _stream(stream)))
        return y

    def pvr_pose_to_fixed(self, pt: PatchTable, poses, fix=None, stream=None):
        if fix is None:
            fix = torch.empty((pt.n, 16), dtype=torch.int32, device=poses.device)
        self._chk(lib.pvr_pose_to_fixed(self.h, C.byref(pt.c), _ptr(poses), _ptr(fix), _stream(stream)))
        return fix

    def pvr_simulate(self, x, pt: PatchTable, poses, sim=None, valid=None, stream=None):
        dev = x.device
        if sim is None:
            sim = torch.empty(pt.n_pix, dtype=torch.float32, device=dev)
        if valid is None:
            valid = torch.empty(pt.n_pix, dtype=torch.uint8, device=dev)
        self._chk(lib.pvr_simulate(self.h, _ptr(x), C.byref(pt.c), _ptr(poses), _ptr(sim), _ptr(valid),
                                   _stream(stream)))
        return sim, valid

    def pvr_adjoint(self, pt: PatchTable, poses, r=None, w=None, addon=None, conf=None,
                    accumulate=False, stream=None):
        dev = poses.device
        if addon is None:
            addon = torch.empty(self.vol_shape, dtype=torch.float32, device=dev)
        if conf is None:
            conf = torch.empty(self.vol_shape, dtype=torch.float32, device=dev)
        self._chk(lib.pvr_adjoint(self.h, C.byref(pt.c), _ptr(poses), _ptr(r), _ptr(w), _ptr(addon),
                                  _ptr(conf), int(bool(accumulate)), _stream(stream)))
        return addon, conf

    def pvr_em_weights(self, y, sim, valid, pt: PatchTable, state, mask_in=None, mask_out=None,
                       p=None, w_patch=None, pbar=None, stream=None):
        dev = y.device
        if mask_out is None:
            mask_out = torch.empty(pt.n, dtype=torch.uint8, device=dev)
        if p is None:
            p = torch.empty(pt.n_pix, dtype=torch.float32, device=dev)
        if w_patch is None:
            w_patch = torch.empty(pt.n, dtype=torch.float32, device=dev)
        if pbar is None:
            pbar = torch.empty(pt.n, dtype=torch.float32, device=dev)
        self._chk(lib.pvr_em_weights(self.h, _ptr(y), _ptr(sim), _ptr(valid), C.byref(pt.c),
                                     _ptr(state), _ptr(mask_in), _ptr(mask_out), _ptr(p),
                                     _ptr(w_patch), _ptr(pbar), _stream(stream)))
        return p, w_patch, pbar, mask_out

    def pvr_volume_update(self, x, addon, conf, clear=True, stream=None):
        self._chk(lib.pvr_volume_update(self.h, _ptr(x), _ptr(addon), _ptr(conf), int(bool(clear)),
                                        _stream(stream)))
        return x

    def pvr_volume_init(self, y, pt: PatchTable, poses, x=None, stream=None):
        if x is None:
            x = torch.empty(self.vol_shape, dtype=torch.float32, device=y.device)
        self._chk(lib.pvr_volume_init(self.h, _ptr(x), _ptr(y), C.byref(pt.c), _ptr(poses),
                                      _stream(stream)))
        return x

    def pvr_ncc_grad(self, x, y, pt: PatchTable, poses, ncc=None, grad=None, want_grad=True,
                     stream=None):
        dev = x.device
        if ncc is None:
            ncc = torch.empty(pt.n, dtype=torch.float64, device=dev)
        if grad is None and want_grad:
            grad = torch.empty((pt.n, self.n_params), dtype=torch.float64, device=dev)
        self._chk(lib.pvr_ncc_grad(self.h, _ptr(x), _ptr(y), C.byref(pt.c), _ptr(poses), _ptr(ncc),
                                   _ptr(grad), _stream(stream)))
        return ncc, grad

    def pvr_patch_metrics(self, y, sim, valid, pt: PatchTable, w=3, want_map=True, stream=None):
        """Per-patch {PSNR, CC, SSIM, DSSIM, mean local SSIM} (float64 [n, 5])
        and the local DSSIM heat map (float32 [n_pix] or None)."""
        out = torch.empty((pt.n, 5), dtype=torch.float64, device=y.device)
        m = torch.empty(pt.n_pix, dtype=torch.float32, device=y.device) if want_map else None
        self._chk(lib.pvr_patch_metrics(self.h, _ptr(y), _ptr(sim), _ptr(valid), C.byref(pt.c), int(w), _ptr(out),
                                        _ptr(m), _stream(stream)))
        return out, m

    def pvr_rigidity_map(self, pt: PatchTable, poses, p, pbar, out=None, stream=None):
        """A^T(p * p-bar) / A^T 1: the rigidity / data-consistency volume."""
        if out is None:
            out = torch.empty(self.vol_shape, dtype=torch.float32, device=poses.device)
        self._chk(lib.pvr_rigidity_map(self.h, C.byref(pt.c), _ptr(poses), _ptr(p), _ptr(pbar), _ptr(out),
                                       _stream(stream)))
        return out

    def pvr_pose_grad(self, x, r, pt: PatchTable, poses, grad=None, stream=None):
        """d (sum_pix r * sim) / d pose per patch (float64 [n, n_params])."""
        if grad is None:
            grad = torch.empty((pt.n, self.n_params), dtype=torch.float64, device=x.device)
        self._chk(lib.pvr_pose_grad(self.h, _ptr(x), _ptr(r), C.byref(pt.c), _ptr(poses), _ptr(grad),
                                    _stream(stream)))
        return grad

    def pvr_plan(self, pt: PatchTable, x=None, y=None, poses=None, tile=0, mode=-1, stream=None):
        """Work plan for this table (tile 0 / mode -1: tuned on x, y, poses);
        returns (tile, mode, n_items)."""
        self._chk(lib.pvr_plan(self.h, C.byref(pt.c), _ptr(x), _ptr(y), _ptr(poses), int(tile), int(mode),
                               _stream(stream)))
        return self.pvr_plan_info()

    def pvr_plan_info(self):
        t, m, n = C.c_int32(0), C.c_int32(0), C.c_int32(0)
        self._chk(lib.pvr_plan_info(self.h, C.byref(t), C.byref(m), C.byref(n)))
        return int(t.value), int(m.value), int(n.value)

    def pvr_plan_order(self, n, stream=None):
        """The plan's patch launch order (numpy int32 [n])."""
        out = np.zeros(max(int(n), 1), dtype=np.int32)
        self._chk(lib.pvr_plan_order(self.h, out.ctypes.data_as(C.c_void_p), int(n), _stream(stream)))
        return out[:int(n)]

    def pvr_plan_clear(self):
        self._chk(lib.pvr_plan_clear(self.h))

    def pvr_graph_capture(self, x, y, pt: PatchTable, poses, state, mask, p=None, w_patch=None,
                          stream=None):
        self._graph_keep = (x, y, pt, poses, state, mask, p, w_patch)   # pointers baked into the graph
        self._chk(lib.pvr_graph_capture(self.h, _ptr(x), _ptr(y), C.byref(pt.c), _ptr(poses), _ptr(state),
                                        _ptr(mask), _ptr(p), _ptr(w_patch), _stream(stream)))

    def pvr_graph_launch(self, stream=None):
        self._chk(lib.pvr_graph_launch(self.h, _stream(stream)))

    def pvr_register(self, x, y, pt: PatchTable, poses, n_evals, ncc=None, stream=None):
        if ncc is None:
            ncc = torch.empty(pt.n, dtype=torch.float64, device=x.device)
        self._chk(lib.pvr_register(self.h, _ptr(x), _ptr(y), C.byref(pt.c), _ptr(poses),
                                   int(n_evals), _ptr(ncc), _stream(stream)))
        return poses, ncc

    def pvr_reconstruct_iter(self, x, y, pt: PatchTable, poses, state, mask, p=None, w_patch=None,
                             stream=None):
        self._chk(lib.pvr_reconstruct_iter(self.h, _ptr(x), _ptr(y), C.byref(pt.c), _ptr(poses),
                                           _ptr(state), _ptr(mask), _ptr(p), _ptr(w_patch),
                                           _stream(stream)))
        return x

    def pvr_profile_enable(self, enable=True):
        self._chk(lib.pvr_profile_enable(self.h, int(bool(enable))))

    def pvr_profile_read(self, stream=None):
        """{class: (ms, launch groups)} since the last read (synchronises)."""
        ms = (C.c_double * len(KERNEL_CLASSES))()
        n = (C.c_int64 * len(KERNEL_CLASSES))()
        self._chk(lib.pvr_profile_read(self.h, ms, n, _stream(stream)))
        return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_CLASSES)}

    def pvr_metrics(self, ref, img, mask=None, out=None, stream=None):
        if out is None:
            out = torch.empty(5, dtype=torch.float64, device=ref.device)
        self._chk(lib.pvr_metrics(self.h, _ptr(ref), _ptr(img), _ptr(mask), int(ref.numel()), _ptr(out),
                                  _stream(stream)))
        return out


class Net:
    """pvr_net: the learned pose proposal CNN (float32 master weights,
    bfloat16 tensor-core convolutions)."""

    def __init__(self, batch_max=256, seed=0):
        h = C.c_void_p()
        rc = lib.pvr_net_create(C.byref(h), int(batch_max), int(seed))
        if rc != 0:
            raise PvrError(rc, "pvr_net_create failed")
        self.h, self.batch_max = h, int(batch_max)

    def __del__(self):
        if getattr(self, "h", None):
            lib.pvr_net_destroy(self.h)
            self.h = None

    def _chk(self, rc, what):
        if rc != 0:
            raise PvrError(rc, what)

    def param_count(self):
        return int(lib.pvr_net_param_count(self.h))

    def get_params(self):
        a = np.zeros(self.param_count(), dtype=np.float32)
        self._chk(lib.pvr_net_get_params(self.h, a.ctypes.data), "pvr_net_get_params")
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        assert a.size == self.param_count()
        self._chk(lib.pvr_net_set_params(self.h, a.ctypes.data), "pvr_net_set_params")

    def get_grads(self):
        a = np.zeros(self.param_count(), dtype=np.float32)
        self._chk(lib.pvr_net_get_grads(self.h, a.ctypes.data), "pvr_net_get_grads")
        return a

    def forward(self, y, s, valid, pt: PatchTable, first=0, count=None, out=None, stream=None):
        count = pt.n - first if count is None else count
        if out is None:
            out = torch.empty((count, 6), dtype=torch.float32, device=y.device)
        self._chk(lib.pvr_net_forward(self.h, _ptr(y), _ptr(s), _ptr(valid), C.byref(pt.c), int(first), int(count),
                                      _ptr(out), _stream(stream)), "pvr_net_forward")
        return out

    def status(self, stream=None):
        """Raise if a bounded wait of a tensor-core convolution gave up."""
        self._chk(lib.pvr_net_status(self.h, _stream(stream)), "pvr_net_status")

    def reserve(self, max_patches, max_pixels):
        self._chk(lib.pvr_net_reserve(self.h, int(max_patches), int(max_pixels)), "pvr_net_reserve")

    def propose(self, ctx: "Context", x, y, pt: PatchTable, poses, scale, accepted=None, stream=None):
        """In place on poses: the network's correction where it raises NCC."""
        sc = (C.c_double * 6)(*[float(v) for v in scale])
        self._chk(lib.pvr_pose_propose(ctx.h, self.h, _ptr(x), _ptr(y), C.byref(pt.c), sc, _ptr(poses),
                                       _ptr(accepted), _stream(stream)), "pvr_pose_propose")
        return poses

    def train_step(self, y, s, valid, pt: PatchTable, first, count, target, lr, loss=None, stream=None):
        self._chk(lib.pvr_net_train_step(self.h, _ptr(y), _ptr(s), _ptr(valid), C.byref(pt.c), int(first),
                                         int(count), _ptr(target), float(lr), _ptr(loss), _stream(stream)),
                  "pvr_net_train_step")
        return loss


def pvr_simulate_noalloc(geom, params: Params, x, pt: PatchTable, poses, sim, valid, stream=None):
    """Context-free pvr_simulate that allocates nothing (see include/pvr.h):
    for callers that cannot allocate device memory.  sim and valid must be
    caller-provided tensors; returns the pvr_status code."""
    g = geometry(geom) if not isinstance(geom, Geometry) else geom
    return int(lib.pvr_simulate_noalloc(C.byref(g), C.byref(params), _ptr(x), C.byref(pt.c),
                                        _ptr(poses), _ptr(sim), _ptr(valid), _stream(stream)))


def pvr_noalloc_status(stream=None):
    """Read and clear the error word of pvr_simulate_noalloc on the current
    device (synchronises); returns the pvr_status code."""
    return int(lib.pvr_noalloc_status(_stream(stream)))


def new_state(device="cuda"):
    return torch.zeros(EM_STATE_LEN, dtype=torch.float64, device=device)
