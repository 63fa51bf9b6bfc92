"""Seeded synthetic inputs for the PVR hot path.

This module only makes inputs: analytic ellipsoid phantoms, acquisition
geometry, slice motion, acquired stacks (analytic phantom integrated under a
dense in-plane x through-plane quadrature, Rician noise, corrupted slices)
and random volumes / poses for small unit cases.  It holds none of the
method's arithmetic (no trilinear sampling of voxel grids, no fixed-point
lattice, no EM, no registration), so both the CUDA path and the CPU oracle
can take their inputs from it.

The paper's data (Brainweb, private fetal MRI) are not available; the two
workloads here stand in for its whole-uterus scans:

* ``config_tiny``: 64^3 voxels of 1 mm, nested ellipsoids (intensities
  0..1000, seeded radii), 3 orthogonal stacks of 20 slices of 64x64 pixels at
  1x1x3 mm, per-slice rigid motion (rotation +-5 deg, translation +-3 mm),
  Rician noise sigma = 2 % of the maximum, square patches 32 / stride 16.
* ``config_uterus``: 256x256x192 voxels of 0.75 mm, maternal body, uterus,
  amniotic fluid, placenta and fetus (body, head, brain), 3 orthogonal + 1
  oblique (30 deg) stacks of 96 slices of 256x256 pixels at 0.75x0.75x2.5 mm,
  breathing motion (8 mm sinusoid, random phase per slice, amplitude linear
  across the field of view: an affine motion per slice), three sudden rigid
  jumps (+-15 deg) of the fetus only, 5 % corrupted slices (half zeroed,
  half scaled by 0.3), patches 64 / stride 32 kept when at least half their
  pixels exceed 1 % of the maximum.
* ``config_uneven``: the uterus volume and stacks with a patch side drawn
  per slice from {32, 48, 64, 96, 128}, stride half the side (batched
  patches of uneven sizes).
* ``config_skew``: interleaved motion-free and skewed slices (the skew
  motion model of the paper's adult-brain experiment) of a nested-ellipsoid
  phantom, three orthogonal stacks.
* ``config_diff``: the differentiable-forward-model workload, 128^3 voxels
  of 1 mm with nested ellipsoids, 3 orthogonal stacks of 86 slices of
  128x128 pixels at 1x1x1.5 mm, all square patches 48 / stride 24 (4,128
  patches of 48x48).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch


@dataclasses.dataclass
class Geometry:
    """Volume grid and stack geometry.

    vol_dims: (nx, ny, nz); the volume is stored [nz][ny][nx], x fastest.
    w2v: 3x4 affine, world (mm) -> voxel index (voxel centres at integers).
    v2w: 3x4 affine, voxel index -> world.
    stack_dims: per stack (W, H, K): columns, rows, slices; stored [K][H][W].
    p2w: per stack 3x4 affine, pixel (column, row, slice) -> world (mm).
    thickness: per stack slice thickness (through-plane FWHM), mm.
    """
    vol_dims: tuple
    w2v: np.ndarray
    v2w: np.ndarray
    stack_dims: list
    p2w: list
    thickness: list

    @property
    def n_vox(self) -> int:
        nx, ny, nz = self.vol_dims
        return nx * ny * nz

    def stack_offsets(self):
        offs, o = [], 0
        for (W, H, K) in self.stack_dims:
            offs.append(o)
            o += W * H * K
        return offs, o


@dataclasses.dataclass
class Ellipsoid:
    centre: np.ndarray
    radii: np.ndarray
    rot: np.ndarray  # 3x3, columns = ellipsoid axes in world
    value: float
    group: str = "static"  # "static" or "fetus"


def rot_zyx(rx, ry, rz):
    """Rz(rz) Ry(ry) Rx(rx), angles in degrees (same convention as the
    rigid pose parameters)."""
    ax, ay, az = (math.radians(v) for v in (rx, ry, rz))
    Rx = np.array([[1, 0, 0], [0, math.cos(ax), -math.sin(ax)], [0, math.sin(ax), math.cos(ax)]])
    Ry = np.array([[math.cos(ay), 0, math.sin(ay)], [0, 1, 0], [-math.sin(ay), 0, math.cos(ay)]])
    Rz = np.array([[math.cos(az), -math.sin(az), 0], [math.sin(az), math.cos(az), 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def volume_geometry(dims, spacing):
    nx, ny, nz = dims
    s = float(spacing)
    ctr = [(nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0]
    v2w = np.zeros((3, 4))
    w2v = np.zeros((3, 4))
    for a in range(3):
        v2w[a, a] = s
        v2w[a, 3] = -ctr[a] * s
        w2v[a, a] = 1.0 / s
        w2v[a, 3] = ctr[a]
    return w2v, v2w


def stack_matrix(u, v, n, W, H, K, sxy, sz, centre=(0.0, 0.0, 0.0)):
    """Pixel -> world for a stack with in-plane unit axes u (columns), v
    (rows) and slice normal n, centred on `centre`."""
    u, v, n = (np.asarray(a, dtype=np.float64) for a in (u, v, n))
    M = np.zeros((3, 4))
    M[:, 0] = u * sxy
    M[:, 1] = v * sxy
    M[:, 2] = n * sz
    M[:, 3] = (np.asarray(centre) - u * sxy * (W - 1) / 2.0 - v * sxy * (H - 1) / 2.0
               - n * sz * (K - 1) / 2.0)
    return M


def pixel_world(p2w, W, H, k):
    """World coordinates of the pixel centres of slice k: array [H, W, 3]."""
    jj, ii = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    return ii[..., None] * p2w[:, 0] + jj[..., None] * p2w[:, 1] + k * p2w[:, 2] + p2w[:, 3]


# --------------------------------------------------------------- phantoms --

def _eval_ellipsoids(pts, ells, fetus_inv=None):
    """Painter's evaluation of ellipsoids at world points pts (torch [N, 3],
    float64).  fetus_inv: optional (R3x3, t3) applied to points before the
    fetus ellipsoids are tested (the inverse of the fetus motion)."""
    val = torch.zeros(pts.shape[0], dtype=pts.dtype, device=pts.device)
    pf = pts
    if fetus_inv is not None:
        R, t = fetus_inv
        pf = pts @ torch.as_tensor(R.T, dtype=pts.dtype, device=pts.device) + torch.as_tensor(
            t, dtype=pts.dtype, device=pts.device)
    for e in ells:
        p = pf if e.group == "fetus" else pts
        c = torch.as_tensor(e.centre, dtype=pts.dtype, device=pts.device)
        Rt = torch.as_tensor(e.rot, dtype=pts.dtype, device=pts.device)
        r = torch.as_tensor(e.radii, dtype=pts.dtype, device=pts.device)
        loc = ((p - c) @ Rt) / r
        inside = (loc * loc).sum(-1) <= 1.0
        val = torch.where(inside, torch.full_like(val, e.value), val)
    return val


def phantom_nested(rng, fov_mm):
    """Nested ellipsoids with seeded radii, intensities within 0..1000."""
    h = fov_mm / 2.0
    ells = []
    specs = [(0.85, 300.0), (0.62, 600.0), (0.38, 900.0)]
    base = np.array([1.0, 0.86, 0.78])
    for frac, val in specs:
        radii = h * frac * base * rng.uniform(0.9, 1.1, 3)
        centre = rng.uniform(-0.04, 0.04, 3) * h
        rot = rot_zyx(*rng.uniform(-15, 15, 3))
        ells.append(Ellipsoid(centre, radii, rot, val))
    for val in (120.0, 1000.0):
        radii = h * rng.uniform(0.10, 0.18, 3)
        centre = rng.uniform(-0.3, 0.3, 3) * h
        ells.append(Ellipsoid(centre, radii, rot_zyx(*rng.uniform(-40, 40, 3)), val))
    return ells


def phantom_uterus(rng):
    """Maternal body, uterus, amniotic fluid, placenta cap and fetus (body,
    head, brain); mm, centred at the origin, fits a 192x192x144 mm box."""
    j = lambda s: rng.uniform(1 - s, 1 + s, 3)
    R0 = rot_zyx(*rng.uniform(-5, 5, 3))
    ells = [
        Ellipsoid(np.array([0.0, 0.0, 0.0]), np.array([90.0, 76.0, 66.0]) * j(0.03), R0, 250.0),
        Ellipsoid(np.array([0.0, 8.0, 0.0]), np.array([68.0, 56.0, 52.0]) * j(0.05), R0, 420.0),
        Ellipsoid(np.array([0.0, 8.0, 0.0]), np.array([61.0, 49.0, 45.0]) * j(0.05), R0, 950.0),
        Ellipsoid(np.array([0.0, 50.0, 5.0]), np.array([44.0, 11.0, 38.0]) * j(0.08),
                  rot_zyx(*rng.uniform(-10, 10, 3)), 560.0),
        Ellipsoid(np.array([-10.0, 0.0, -8.0]), np.array([30.0, 18.0, 20.0]) * j(0.08),
                  rot_zyx(*rng.uniform(-20, 20, 3)), 460.0, "fetus"),
        Ellipsoid(np.array([24.0, -2.0, 6.0]), np.array([17.0, 14.0, 15.0]) * j(0.05),
                  rot_zyx(*rng.uniform(-20, 20, 3)), 310.0, "fetus"),
        Ellipsoid(np.array([24.5, -2.0, 6.0]), np.array([13.5, 10.5, 11.5]) * j(0.05),
                  rot_zyx(*rng.uniform(-20, 20, 3)), 720.0, "fetus"),
    ]
    fetus_centre = np.array([8.0, -1.0, -2.0])
    return ells, fetus_centre


def ground_truth(ells, geom: Geometry, device="cpu"):
    """Unmoved phantom sampled at the voxel centres: float32 [nz, ny, nx]."""
    nx, ny, nz = geom.vol_dims
    out = torch.empty((nz, ny, nx), dtype=torch.float32)
    v2w = torch.as_tensor(geom.v2w, dtype=torch.float64, device=device)
    yy, xx = torch.meshgrid(torch.arange(ny, dtype=torch.float64, device=device),
                            torch.arange(nx, dtype=torch.float64, device=device), indexing="ij")
    for z in range(nz):
        vox = torch.stack([xx, yy, torch.full_like(xx, float(z))], -1).reshape(-1, 3)
        pts = vox @ v2w[:, :3].T + v2w[:, 3]
        out[z] = _eval_ellipsoids(pts, ells).reshape(ny, nx).float().cpu()
    return out


# ------------------------------------------------------------ acquisition --

def _quadrature(fwhm_xy_px, thick_mm, sz_mm):
    """In-plane 3x3 points at +-0.5 px and 5 through-plane points over
    +-2 sigma_z, Gaussian weights normalised to 1.  Returns (offsets [Q, 3] in
    (px, px, slice units), weights [Q])."""
    sxy = fwhm_xy_px / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    szm = thick_mm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    offs, wts = [], []
    for dj in (-0.5, 0.0, 0.5):
        for di in (-0.5, 0.0, 0.5):
            for t in (-2.0, -1.0, 0.0, 1.0, 2.0):
                dz_mm = t * szm
                w = math.exp(-(di * di + dj * dj) / (2 * sxy * sxy)) * math.exp(-(t * t) / 2.0)
                offs.append((di, dj, dz_mm / sz_mm))
                wts.append(w)
    wts = np.array(wts)
    return np.array(offs), wts / wts.sum()


def acquire(ells, geom: Geometry, motion, rng, noise_sigma, fwhm_xy_px=1.2, device="cpu",
            fetus_motion=None, corrupt=None):
    """Acquire every stack from the analytic phantom.

    motion(s, k) -> (L 3x3, b 3): affine map scanner world -> anatomy for
    slice k of stack s.  fetus_motion(s, k) -> (R, t) inverse fetus motion
    or None.  corrupt: dict {(s, k): factor}.  Returns a list of float32
    arrays [K, H, W]."""
    out = []
    gen = torch.Generator(device="cpu").manual_seed(int(rng.integers(0, 2**31 - 1)))
    for s, (W, H, K) in enumerate(geom.stack_dims):
        p2w = np.asarray(geom.p2w[s])
        sz_mm = float(np.linalg.norm(p2w[:, 2]))
        offs, wts = _quadrature(fwhm_xy_px, geom.thickness[s], sz_mm)
        wts_t = torch.as_tensor(wts, dtype=torch.float64, device=device)
        M = torch.as_tensor(p2w, dtype=torch.float64, device=device)
        jj, ii = torch.meshgrid(torch.arange(H, dtype=torch.float64, device=device),
                                torch.arange(W, dtype=torch.float64, device=device), indexing="ij")
        stack = torch.empty((K, H, W), dtype=torch.float32)
        for k in range(K):
            L, b = motion(s, k)
            Lt = torch.as_tensor(L, dtype=torch.float64, device=device)
            bt = torch.as_tensor(b, dtype=torch.float64, device=device)
            acc = torch.zeros((H, W), dtype=torch.float64, device=device)
            fm = fetus_motion(s, k) if fetus_motion is not None else None
            for q in range(offs.shape[0]):
                px = torch.stack([ii + offs[q, 0], jj + offs[q, 1],
                                  torch.full_like(ii, k + offs[q, 2])], -1).reshape(-1, 3)
                w = px @ M[:, :3].T + M[:, 3]
                a = w @ Lt.T + bt
                acc += wts_t[q] * _eval_ellipsoids(a, ells, fm).reshape(H, W)
            img = acc.cpu()
            if noise_sigma > 0:
                n1 = torch.randn((H, W), generator=gen, dtype=torch.float64) * noise_sigma
                n2 = torch.randn((H, W), generator=gen, dtype=torch.float64) * noise_sigma
                img = torch.sqrt((img + n1) ** 2 + n2 ** 2)
            if corrupt is not None and (s, k) in corrupt:
                img = img * corrupt[(s, k)]
            stack[k] = img.float()
        out.append(stack.numpy())
    return out


def pack_stacks(stacks):
    return np.concatenate([np.ascontiguousarray(s, dtype=np.float32).reshape(-1) for s in stacks])


def pack_patch_pixels(stacks, desc):
    """Patch pixels, patch after patch, row-major within a patch (pure
    indexing of the acquired stacks)."""
    n = int(sum(int(d[4]) * int(d[5]) for d in desc))
    y = np.empty(n, dtype=np.float32)
    for d in desc:
        s, k, x0, y0, w, h, off = (int(v) for v in d[:7])
        y[off:off + w * h] = stacks[s][k, y0:y0 + h, x0:x0 + w].reshape(-1)
    return y


def rigid_patch_poses(geom: Geometry, desc, slice_rot, slice_t):
    """Per-patch rigid parameters (tx, ty, tz mm; rx, ry, rz deg) of a slice
    motion T(w) = R (w - c_k) + c_k + t_k (c_k the slice centre) re-expressed
    about each patch centre c_p: t_p = t_k + (R - I)(c_p - c_k)."""
    poses = np.zeros((len(desc), 6))
    for n, d in enumerate(desc):
        s, k, x0, y0, w, h = (int(v) for v in d[:6])
        W, H, K = geom.stack_dims[s]
        p2w = np.asarray(geom.p2w[s])
        ck = p2w[:, 0] * (W - 1) / 2 + p2w[:, 1] * (H - 1) / 2 + p2w[:, 2] * k + p2w[:, 3]
        cp = p2w[:, 0] * (x0 + (w - 1) / 2) + p2w[:, 1] * (y0 + (h - 1) / 2) + p2w[:, 2] * k + p2w[:, 3]
        ang = slice_rot[s][k]
        R = rot_zyx(*ang)
        poses[n, :3] = slice_t[s][k] + (R - np.eye(3)) @ (cp - ck)
        poses[n, 3:] = ang
    return poses


# ---------------------------------------------------------------- configs --

def config_tiny(seed=1611, device="cpu", noise=True):
    """64^3 nested-ellipsoid workload (see module docstring)."""
    rng = np.random.default_rng(seed)
    dims, sp = (64, 64, 64), 1.0
    w2v, v2w = volume_geometry(dims, sp)
    W = H = 64
    K = 20
    axes = [((1, 0, 0), (0, 1, 0), (0, 0, 1)),
            ((1, 0, 0), (0, 0, 1), (0, 1, 0)),
            ((0, 1, 0), (0, 0, 1), (1, 0, 0))]
    p2w = [stack_matrix(u, v, n, W, H, K, 1.0, 3.0) for (u, v, n) in axes]
    geom = Geometry(dims, w2v, v2w, [(W, H, K)] * 3, p2w, [3.0, 3.0, 3.0])
    ells = phantom_nested(rng, 64.0)
    slice_rot = [rng.uniform(-5, 5, (K, 3)) for _ in range(3)]
    slice_t = [rng.uniform(-3, 3, (K, 3)) for _ in range(3)]

    def motion(s, k):
        R = rot_zyx(*slice_rot[s][k])
        ck = p2w[s][:, 0] * (W - 1) / 2 + p2w[s][:, 1] * (H - 1) / 2 + p2w[s][:, 2] * k + p2w[s][:, 3]
        return R, ck + slice_t[s][k] - R @ ck

    stacks = acquire(ells, geom, motion, rng, 20.0 if noise else 0.0, device=device)
    gt = ground_truth(ells, geom, device=device)
    return dict(name="tiny-64", geom=geom, stacks=stacks, gt=gt.numpy(), ellipsoids=ells,
                slice_rot=slice_rot, slice_t=slice_t, a=32, stride=16, fg_frac=0.0, keep_frac=0.0,
                fwhm_xy=1.2, dz=sp, n_outer=3)


def config_uterus(seed=7289, device="cpu", slices=96, size=256):
    """Whole-uterus workload (see module docstring)."""
    rng = np.random.default_rng(seed)
    dims, sp = (256, 256, 192), 0.75
    w2v, v2w = volume_geometry(dims, sp)
    W = H = size
    K = slices
    c30, s30 = math.cos(math.radians(30)), math.sin(math.radians(30))
    axes = [((1, 0, 0), (0, 1, 0), (0, 0, 1)),
            ((1, 0, 0), (0, 0, 1), (0, 1, 0)),
            ((0, 1, 0), (0, 0, 1), (1, 0, 0)),
            ((1, 0, 0), (0, c30, s30), (0, -s30, c30))]
    sxy = 0.75 * 256 / size
    p2w = [stack_matrix(u, v, n, W, H, K, sxy, 2.5) for (u, v, n) in axes]
    geom = Geometry(dims, w2v, v2w, [(W, H, K)] * 4, p2w, [2.5] * 4)
    ells, fetus_centre = phantom_uterus(rng)
    phase = [rng.uniform(0, 2 * math.pi, K) for _ in range(4)]
    n_total = 4 * K
    jumps = sorted(rng.choice(np.arange(1, n_total), size=3, replace=False).tolist())
    jump_rot = [rot_zyx(*rng.uniform(-15, 15, 3)) for _ in range(3)]
    jump_t = [rng.uniform(-3, 3, 3) for _ in range(3)]
    poses_f = []
    Rf, tf = np.eye(3), np.zeros(3)
    jj = 0
    for t in range(n_total):
        while jj < 3 and t >= jumps[jj]:
            # the fetus occupies Rf (p - c) + c + tf; a jump rotates it about
            # its current centre c + tf and shifts it: Rf <- Rn Rf, tf <- tf + jt
            Rf = jump_rot[jj] @ Rf
            tf = tf + jump_t[jj]
            jj += 1
        poses_f.append((Rf.copy(), tf.copy()))
    n_bad = max(1, int(round(0.05 * n_total)))
    bad = rng.choice(np.arange(n_total), size=n_bad, replace=False)
    corrupt = {}
    for i, b in enumerate(sorted(bad.tolist())):
        corrupt[(b // K, b % K)] = 0.0 if i % 2 == 0 else 0.3

    def motion(s, k):
        amp = 8.0 * math.sin(phase[s][k])
        # displacement along y, amplitude linear across the field of view in y
        L = np.eye(3)
        L[1, 1] += amp / 192.0
        b = np.array([0.0, amp * 0.5, 0.0])
        return L, b

    def fetus_motion(s, k):
        Rf_, tf_ = poses_f[s * K + k]
        # fetus occupies R (p - c) + c + t; inverse map p -> R^T (p - c - t) + c
        Ri = Rf_.T
        return Ri, fetus_centre - Ri @ (fetus_centre + tf_)

    stacks = acquire(ells, geom, motion, rng, 20.0, device=device, fetus_motion=fetus_motion,
                     corrupt=corrupt)
    gt = ground_truth(ells, geom, device=device)
    return dict(name="uterus-256x256x192", geom=geom, stacks=stacks, gt=gt.numpy(),
                ellipsoids=ells, corrupt=corrupt, a=64, stride=32, fg_frac=0.01, keep_frac=0.5,
                fwhm_xy=1.2, dz=sp, n_outer=10)


def uneven_sides(cfg, seed=7289, sides=(32, 48, 64, 96, 128)):
    """A copy of a workload dictionary with a patch side per slice drawn from
    `sides` and stride side / 2 (slice_a, slice_stride: one entry per slice
    of every stack, in order)."""
    rng = np.random.default_rng(seed + 1)
    nk = sum(k for (_, _, k) in cfg["geom"].stack_dims)
    sa = rng.choice(np.asarray(sides, dtype=np.int32), nk).astype(np.int32)
    out = dict(cfg)
    out.update(name=cfg["name"] + "-uneven", slice_a=sa, slice_stride=(sa // 2).astype(np.int32))
    return out


def config_uneven(seed=7289, device="cpu", slices=96, size=256, sides=(32, 48, 64, 96, 128)):
    """Uterus workload with a patch side per slice (module docstring): the
    config_uterus dictionary plus slice_a, slice_stride (one entry per slice
    of every stack, in order)."""
    return uneven_sides(config_uterus(seed=seed, device=device, slices=slices, size=size), seed, sides)


def skew_matrix(theta_deg):
    """The skew (shear) motion of the paper's adult-brain experiment (Sec. IV):
    ones on the diagonal and S = tan(theta) off the diagonal."""
    S = math.tan(math.radians(theta_deg))
    return np.array([[1.0, S, S], [S, 1.0, S], [S, S, 1.0]])


def config_skew(theta_deg=5.0, seed=1283, device="cpu", n=96, spacing=1.25, noise=0.0):
    """Skew-motion workload after the paper's adult-brain study (data not
    available, a nested-ellipsoid phantom instead): n^3 voxels of `spacing`
    mm, axial / coronal / sagittal stacks of n x n pixels at spacing x
    spacing x 2 spacing mm whose slices alternate between the motion-free
    phantom (even slices) and the phantom skewed by skew_matrix(theta)
    about its centre (odd slices), as interleaved acquisition would give."""
    rng = np.random.default_rng(seed)
    dims = (n, n, n)
    w2v, v2w = volume_geometry(dims, spacing)
    K = n // 2
    axes = [((1, 0, 0), (0, 1, 0), (0, 0, 1)),
            ((1, 0, 0), (0, 0, 1), (0, 1, 0)),
            ((0, 1, 0), (0, 0, 1), (1, 0, 0))]
    p2w = [stack_matrix(u, v, w, n, n, K, spacing, 2 * spacing) for (u, v, w) in axes]
    geom = Geometry(dims, w2v, v2w, [(n, n, K)] * 3, p2w, [2 * spacing] * 3)
    ells = phantom_nested(rng, n * spacing)
    T = skew_matrix(theta_deg)
    Ti = np.linalg.inv(T)

    def motion(s, k):
        # the phantom occupies T p in skewed slices; acquisition maps the
        # scanner point p to the anatomy point T^-1 p
        return (Ti, np.zeros(3)) if k % 2 else (np.eye(3), np.zeros(3))

    stacks = acquire(ells, geom, motion, rng, noise, device=device)
    gt = ground_truth(ells, geom, device=device)
    return dict(name=f"skew-{theta_deg}deg", geom=geom, stacks=stacks, gt=gt.numpy(), ellipsoids=ells,
                skew=T, a=32, stride=16, fg_frac=0.01, keep_frac=0.5, fwhm_xy=1.2, dz=spacing)


def config_diff(seed=3, device="cpu"):
    """128^3 workload of the differentiable forward model (module docstring):
    geometry, ground-truth volume and the full patch table."""
    rng = np.random.default_rng(seed)
    dims, sp = (128, 128, 128), 1.0
    w2v, v2w = volume_geometry(dims, sp)
    W = H = 128
    K = 86
    axes = [((1, 0, 0), (0, 1, 0), (0, 0, 1)),
            ((1, 0, 0), (0, 0, 1), (0, 1, 0)),
            ((0, 1, 0), (0, 0, 1), (1, 0, 0))]
    p2w = [stack_matrix(u, v, n, W, H, K, 1.0, 1.5) for (u, v, n) in axes]
    geom = Geometry(dims, w2v, v2w, [(W, H, K)] * 3, p2w, [1.5, 1.5, 1.5])
    ells = phantom_nested(rng, 128.0)
    gt = ground_truth(ells, geom, device=device)
    desc, npix = all_patches(geom, 48, 24)
    return dict(name="diff-128", geom=geom, gt=gt.cpu().numpy(), ellipsoids=ells, desc=desc, n_pix=npix,
                a=48, stride=24, fwhm_xy=1.2, dz=sp)


def random_geometry(rng, n=8, n_stacks=2, W=6, H=5, K=3, spacing=1.0, pix=1.0, thick=2.0):
    """Small geometry with randomly oriented stacks through an n^3 volume
    (unit tests and brute-force checks)."""
    w2v, v2w = volume_geometry((n, n, n), spacing)
    p2w = []
    for _ in range(n_stacks):
        R = rot_zyx(*rng.uniform(-180, 180, 3))
        centre = rng.uniform(-0.5, 0.5, 3) * spacing
        p2w.append(stack_matrix(R[:, 0], R[:, 1], R[:, 2], W, H, K, pix, thick, centre))
    return Geometry((n, n, n), w2v, v2w, [(W, H, K)] * n_stacks, p2w, [thick] * n_stacks)


def all_patches(geom: Geometry, a, stride):
    """Square patch table without foreground rejection (pure enumeration),
    same order and layout as the patch-table builders."""
    rows, off = [], 0
    for s, (W, H, K) in enumerate(geom.stack_dims):
        for k in range(K):
            for y0 in range(0, H - a + 1, stride):
                for x0 in range(0, W - a + 1, stride):
                    rows.append([s, k, x0, y0, a, a, off, 0])
                    off += a * a
    return np.array(rows, dtype=np.int32).reshape(-1, 8), off


def random_poses(rng, P, rot=5.0, trans=3.0):
    return np.concatenate([rng.uniform(-trans, trans, (P, 3)), rng.uniform(-rot, rot, (P, 3))], 1)
