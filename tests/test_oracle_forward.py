"""Pins of the oracle's forward model and adjoint against facts fixed by the
mathematics, independent of the oracle's own code:

* a constant volume simulates to the same constant on every valid pixel;
* identity pose + delta PSF is plain trilinear resampling (scipy's order-1
  map_coordinates at the pixel centres);
* a dense A built column by column from unit volumes equals an independent
  FP64 numpy construction of the PSF-weighted, normalised trilinear operator
  (Eq. 1, W = D B T) -- this fixes the transform convention, the patch
  centre, the through-plane step and the PSF weights;
* the adjoint equals A^T of that dense matrix, and the dot-product test holds
  to 1e-12;
* integer-voxel translations and 90-degree rotations give exact permutations
  of voxel values;
* affine poses (T(w) = (I + D)(w - c) + c + t, 12 parameters): the dense
  operator equals the same independent construction with the linear part
  I + D, D = 0 reproduces the rigid identity lattice bit for bit, and the
  lattice vectors agree with a numpy composition to one Q11.20 quantum.
"""
import math

import numpy as np
import pytest
from scipy.ndimage import map_coordinates
from scipy.spatial.transform import Rotation

from oracle import pvr_oracle as O
from paper_1611_07289_b300 import synth


def _small_case(seed=3, n=8, kxy=1, kz=2, n_stacks=2, a=4, stride=2):
    rng = np.random.default_rng(seed)
    geom = synth.random_geometry(rng, n=n, n_stacks=n_stacks, W=6, H=5, K=3, thick=2.0)
    desc, npix = synth.all_patches(geom, a, stride)
    poses = synth.random_poses(rng, desc.shape[0], rot=5.0, trans=1.0)
    G = O.geom(geom)
    ps = O.psf(1.2, kxy, kz, 1.0)
    return rng, geom, desc, npix, poses, G, ps


def _independent_dense_A(geom, desc, poses, fwhm_xy, kxy, kz, dz):
    """Dense forward operator from plain FP64 linear algebra (no fixed point)."""
    nx, ny, nz = geom.vol_dims
    npix = int(sum(int(d[4]) * int(d[5]) for d in desc))
    A = np.zeros((npix, nx * ny * nz))
    to_sigma = 1.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    sxy = fwhm_xy * to_sigma
    W2V = np.asarray(geom.w2v)
    for d, th in zip(desc, poses):
        s, k, x0, y0, w, h, off = (int(v) for v in d[:7])
        P = np.asarray(geom.p2w[s])
        nrm = P[:, 2] / np.linalg.norm(P[:, 2])
        sz = geom.thickness[s] * to_sigma
        if len(th) == 12:   # affine: linear part I + D, D row-major
            R = np.eye(3) + np.asarray(th[3:12]).reshape(3, 3)
        else:
            R = Rotation.from_euler("ZYX", [th[5], th[4], th[3]], degrees=True).as_matrix()
        c = P @ np.array([x0 + (w - 1) / 2.0, y0 + (h - 1) / 2.0, k, 1.0])
        for j in range(h):
            for i in range(w):
                row = off + j * w + i
                entries = {}
                total = 0.0
                for dj in range(-kxy, kxy + 1):
                    for di in range(-kxy, kxy + 1):
                        for z in range(-kz, kz + 1):
                            wp = P @ np.array([x0 + i + di, y0 + j + dj, k, 1.0]) + nrm * z * dz
                            tw = R @ (wp - c) + c + th[:3]
                            v = W2V[:, :3] @ tw + W2V[:, 3]
                            if np.any(v < 0) or v[0] > nx - 1 or v[1] > ny - 1 or v[2] > nz - 1:
                                continue
                            g = (math.exp(-di * di / (2 * sxy * sxy)) * math.exp(-dj * dj / (2 * sxy * sxy))
                                 * math.exp(-(z * dz) ** 2 / (2 * sz * sz)))
                            total += g
                            b = np.minimum(np.floor(v).astype(int), np.array([nx, ny, nz]) - 2)
                            f = v - b
                            for cz in (0, 1):
                                for cy in (0, 1):
                                    for cx in (0, 1):
                                        wt = ((f[0] if cx else 1 - f[0]) * (f[1] if cy else 1 - f[1])
                                              * (f[2] if cz else 1 - f[2]))
                                        idx = ((b[2] + cz) * ny + b[1] + cy) * nx + b[0] + cx
                                        entries[idx] = entries.get(idx, 0.0) + g * wt
                if total > 0:
                    for idx, val in entries.items():
                        A[row, idx] += val / total
    return A


def test_constant_volume_gives_constant_patches():
    rng, geom, desc, npix, poses, G, ps = _small_case(seed=11, n=10)
    fix = O.pose_fixed(G, ps, desc, poses)
    x = np.full(geom.n_vox, 437.25, dtype=np.float32)
    sim, valid, den = O.simulate(G, ps, x, desc, fix, npix)
    assert valid.sum() > 0.5 * npix
    np.testing.assert_allclose(sim[valid > 0], 437.25, rtol=1e-13)
    assert np.all(sim[valid == 0] == 0.0)
    assert np.all((den > 0) == (valid > 0))


def test_identity_delta_psf_is_trilinear_resampling():
    rng = np.random.default_rng(5)
    n = 12
    geom = synth.random_geometry(rng, n=n, n_stacks=3, W=7, H=7, K=3, thick=1.5)
    desc, npix = synth.all_patches(geom, 7, 7)
    poses = np.zeros((desc.shape[0], 6))
    G = O.geom(geom)
    ps = O.psf(1.2, 0, 0, 1.0)
    fix = O.pose_fixed(G, ps, desc, poses)
    x = rng.uniform(0, 1, geom.n_vox).astype(np.float32)
    sim, valid, _ = O.simulate(G, ps, x, desc, fix, npix)
    vol = x.reshape(n, n, n)  # [z][y][x]
    W2V = np.asarray(geom.w2v)
    checked = 0
    for d in desc:
        s, k, x0, y0, w, h, off = (int(v) for v in d[:7])
        P = np.asarray(geom.p2w[s])
        for j in range(h):
            for i in range(w):
                v = W2V[:, :3] @ (P @ np.array([x0 + i, y0 + j, k, 1.0])) + W2V[:, 3]
                inside = np.all(v >= 0) and np.all(v <= n - 1)
                margin = min(v.min(), (n - 1 - v).min())
                if abs(margin) < 1e-4:
                    continue
                assert bool(valid[off + j * w + i]) == bool(inside)
                if inside:
                    ref = map_coordinates(vol, [[v[2]], [v[1]], [v[0]]], order=1)[0]
                    assert abs(sim[off + j * w + i] - ref) < 5e-6
                    checked += 1
    assert checked > 50


def test_dense_operator_matches_independent_construction():
    rng, geom, desc, npix, poses, G, ps = _small_case(seed=3)
    fix = O.pose_fixed(G, ps, desc, poses)
    nv = geom.n_vox
    A = np.zeros((npix, nv))
    for v in range(nv):
        e = np.zeros(nv, dtype=np.float32)
        e[v] = 1.0
        A[:, v], _, _ = O.simulate(G, ps, e, desc, fix, npix)
    A_ind = _independent_dense_A(geom, desc, poses, 1.2, 1, 2, 1.0)
    assert np.abs(A).sum() > 10.0
    np.testing.assert_allclose(A, A_ind, atol=2e-5)
    # rows of A sum to one on valid pixels (normalised PSF)
    _, valid, _ = O.simulate(G, ps, np.ones(nv, dtype=np.float32), desc, fix, npix)
    np.testing.assert_allclose(A.sum(1)[valid > 0], 1.0, atol=1e-12)
    # the adjoint is A^T
    r = rng.normal(size=npix)
    w = rng.uniform(0, 1, npix)
    addon, conf = O.adjoint(G, ps, desc, fix, r=r, w=w)
    np.testing.assert_allclose(addon, A.T @ (w * r), atol=1e-12)
    np.testing.assert_allclose(conf, A.T @ w, atol=1e-12)


def _affine_poses(rng, n, dmax=0.12, trans=1.0):
    return np.concatenate([rng.uniform(-trans, trans, (n, 3)), rng.uniform(-dmax, dmax, (n, 9))], 1)


def test_affine_dense_operator_matches_independent_construction():
    rng, geom, desc, npix, _, G, ps = _small_case(seed=5)
    poses = _affine_poses(rng, desc.shape[0])
    fix = O.pose_fixed(G, ps, desc, poses, n_params=12)
    nv = geom.n_vox
    A = np.zeros((npix, nv))
    for v in range(nv):
        e = np.zeros(nv, dtype=np.float32)
        e[v] = 1.0
        A[:, v], _, _ = O.simulate(G, ps, e, desc, fix, npix)
    A_ind = _independent_dense_A(geom, desc, poses, 1.2, 1, 2, 1.0)
    assert np.abs(A).sum() > 10.0
    np.testing.assert_allclose(A, A_ind, atol=2e-5)
    # a rigid pose read as affine is a different transform: the poses matter
    fix6 = O.pose_fixed(G, ps, desc, poses[:, :6])
    assert not np.array_equal(fix6[:, :12], fix[:, :12])


def test_affine_identity_equals_rigid_identity_lattice():
    """D = 0 and zero angles both give the linear part I exactly, so the
    lattices agree bit for bit for any translation."""
    rng, geom, desc, npix, _, G, ps = _small_case(seed=6)
    t = rng.uniform(-2, 2, (desc.shape[0], 3))
    rigid = np.concatenate([t, np.zeros((desc.shape[0], 3))], 1)
    affine = np.concatenate([t, np.zeros((desc.shape[0], 9))], 1)
    assert np.array_equal(O.pose_fixed(G, ps, desc, rigid), O.pose_fixed(G, ps, desc, affine, n_params=12))


def test_affine_lattice_matches_numpy_within_one_quantum():
    rng = np.random.default_rng(19)
    geom = synth.random_geometry(rng, n=20, n_stacks=2, W=8, H=8, K=4, thick=2.0)
    desc, _ = synth.all_patches(geom, 4, 4)
    poses = _affine_poses(rng, desc.shape[0], dmax=0.3, trans=3.0)
    G = O.geom(geom)
    ps = O.psf(1.2, 1, 2, 0.7)
    fix = O.pose_fixed(G, ps, desc, poses, n_params=12)
    W2V = np.asarray(geom.w2v)
    for d, th, f in zip(desc, poses, fix):
        P = np.asarray(geom.p2w[int(d[0])])
        L = np.eye(3) + th[3:].reshape(3, 3)
        c = P @ np.array([d[2] + (d[4] - 1) / 2.0, d[3] + (d[5] - 1) / 2.0, d[1], 1.0])
        o = W2V[:, :3] @ (L @ (P @ np.array([d[2], d[3], d[1], 1.0]) - c) + c + th[:3]) + W2V[:, 3]
        ei = W2V[:, :3] @ L @ P[:, 0]
        ej = W2V[:, :3] @ L @ P[:, 1]
        ez = W2V[:, :3] @ L @ (P[:, 2] / np.linalg.norm(P[:, 2]) * 0.7)
        assert f[12] == 1
        for vec, sl in ((o, slice(0, 3)), (ei, slice(3, 6)), (ej, slice(6, 9)), (ez, slice(9, 12))):
            assert np.max(np.abs(np.round(vec * 2**20) - f[sl])) <= 1


@pytest.mark.parametrize("seed", [1, 2])
def test_dot_product_adjoint(seed):
    rng = np.random.default_rng(100 + seed)
    geom = synth.random_geometry(rng, n=16, n_stacks=3, W=14, H=12, K=5, thick=2.5)
    desc, npix = synth.all_patches(geom, 6, 3)
    poses = synth.random_poses(rng, desc.shape[0], rot=8.0, trans=2.0)
    G = O.geom(geom)
    ps = O.psf(1.2, 1, 3, 0.8)
    fix = O.pose_fixed(G, ps, desc, poses)
    x = rng.normal(size=geom.n_vox).astype(np.float32)
    r = rng.normal(size=npix)
    Ax, valid, _ = O.simulate(G, ps, x, desc, fix, npix)
    ATr, _ = O.adjoint(G, ps, desc, fix, r=r, w=None)
    lhs = float(np.dot(Ax, r))
    rhs = float(np.dot(x.astype(np.float64), ATr))
    assert valid.sum() > 100
    assert abs(lhs - rhs) / (np.linalg.norm(Ax) * np.linalg.norm(r)) < 1e-12


def _aligned_geometry(n=16):
    """Axial stack aligned with the voxel grid (1 mm pixels, 1 mm slices)."""
    w2v, v2w = synth.volume_geometry((n, n, n), 1.0)
    P = synth.stack_matrix((1, 0, 0), (0, 1, 0), (0, 0, 1), n, n, n, 1.0, 1.0)
    return synth.Geometry((n, n, n), w2v, v2w, [(n, n, n)], [P], [1.0])


def test_integer_translation_is_exact_shift():
    n = 16
    geom = _aligned_geometry(n)
    G = O.geom(geom)
    ps = O.psf(1.2, 0, 0, 1.0)
    desc = np.array([[0, 6, 4, 5, 6, 4, 0, 0]], dtype=np.int32)
    th = np.array([[2.0, -3.0, 1.0, 0.0, 0.0, 0.0]])
    fix = O.pose_fixed(G, ps, desc, th)
    assert fix[0, 12] == 1
    assert all(v % (1 << 20) == 0 for v in fix[0, :3])
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1000, geom.n_vox).astype(np.float32)
    sim, valid, _ = O.simulate(G, ps, x, desc, fix, 24)
    vol = x.reshape(n, n, n)
    exp = vol[6 + 1, 5 - 3:5 - 3 + 4, 4 + 2:4 + 2 + 6].reshape(-1)
    assert np.all(valid == 1)
    assert np.array_equal(sim, exp.astype(np.float64))


def test_quarter_turns_are_exact_permutations():
    n = 16
    geom = _aligned_geometry(n)
    G = O.geom(geom)
    ps = O.psf(1.2, 0, 0, 1.0)
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1000, geom.n_vox).astype(np.float32)
    vol = x.reshape(n, n, n)
    x0, y0, k, w, h = 4, 6, 7, 6, 6
    desc = np.array([[0, k, x0, y0, w, h, 0, 0]], dtype=np.int32)
    cx, cy = x0 + (w - 1) / 2.0, y0 + (h - 1) / 2.0
    for q in (1, 2, 3, -1, 5):
        th = np.array([[0.0, 0.0, 0.0, 0.0, 0.0, 90.0 * q]])
        fix = O.pose_fixed(G, ps, desc, th)
        sim, valid, _ = O.simulate(G, ps, x, desc, fix, w * h)
        ang = math.radians(90.0 * q)
        cs, sn = round(math.cos(ang)), round(math.sin(ang))
        exp = np.empty(w * h)
        for j in range(h):
            for i in range(w):
                px, py = x0 + i - cx, y0 + j - cy
                vx, vy = cs * px - sn * py + cx, sn * px + cs * py + cy
                exp[j * w + i] = vol[k, int(round(vy)), int(round(vx))]
        assert np.all(valid == 1)
        assert np.array_equal(sim, exp), q


def test_rotation_lattice_matches_libm_within_one_quantum():
    """The fixed-point lattice vectors agree with an FP64 libm evaluation of
    w2v . R . p2w to within one Q11.20 quantum (sin/cos are evaluated from
    their series in the oracle)."""
    rng = np.random.default_rng(9)
    geom = synth.random_geometry(rng, n=20, n_stacks=2, W=8, H=8, K=4, thick=2.0)
    desc, _ = synth.all_patches(geom, 4, 4)
    poses = synth.random_poses(rng, desc.shape[0], rot=170.0, trans=3.0)
    G = O.geom(geom)
    ps = O.psf(1.2, 1, 2, 0.7)
    fix = O.pose_fixed(G, ps, desc, poses)
    W2V = np.asarray(geom.w2v)
    for d, th, f in zip(desc, poses, fix):
        P = np.asarray(geom.p2w[int(d[0])])
        R = Rotation.from_euler("ZYX", [th[5], th[4], th[3]], degrees=True).as_matrix()
        ei = W2V[:, :3] @ R @ P[:, 0]
        ej = W2V[:, :3] @ R @ P[:, 1]
        ez = W2V[:, :3] @ R @ (P[:, 2] / np.linalg.norm(P[:, 2]) * 0.7)
        for vec, sl in ((ei, slice(3, 6)), (ej, slice(6, 9)), (ez, slice(9, 12))):
            assert np.max(np.abs(np.round(vec * 2**20) - f[sl])) <= 1


def test_out_of_range_pose_invalidates_patch():
    rng, geom, desc, npix, poses, G, ps = _small_case(seed=4)
    poses = poses.copy()
    poses[0, 0] = 5.0e3  # 5 m away: beyond the Q11.20 range
    fix = O.pose_fixed(G, ps, desc, poses)
    assert fix[0, 12] == 0 and np.all(fix[0, :12] == 0)
    x = np.ones(geom.n_vox, dtype=np.float32)
    sim, valid, _ = O.simulate(G, ps, x, desc, fix, npix)
    n0 = int(desc[0, 4] * desc[0, 5])
    assert np.all(valid[:n0] == 0)


def test_patch_table_enumeration_and_rejection():
    rng = np.random.default_rng(2)
    geom = synth.random_geometry(rng, n=8, n_stacks=2, W=20, H=12, K=2)
    _, total = geom.stack_offsets()
    stacks = np.zeros(total, dtype=np.float32)
    desc, npix = O.patches_build(O.geom(geom), stacks + 1.0, 8, 4)
    ref, ref_n = synth.all_patches(geom, 8, 4)
    assert np.array_equal(desc, ref) and npix == ref_n
    # one bright 8x8 block in stack 1, slice 0 at (x=4..11, y=4..11): only the
    # patch at (4, 4) has all its pixels above the level
    img = stacks.reshape(-1).copy()
    off1 = 20 * 12 * 2
    for yy in range(4, 12):
        img[off1 + yy * 20 + 4: off1 + yy * 20 + 12] = 100.0
    desc2, npix2 = O.patches_build(O.geom(geom), img, 8, 4, fg_frac=0.01, keep_frac=1.0)
    assert desc2.shape[0] == 1 and list(desc2[0, :7]) == [1, 0, 4, 4, 8, 8, 0] and npix2 == 64


def test_multi_size_patch_table_enumeration_and_rejection():
    """Per-slice sizes: without rejection the table is the plain enumeration
    (written out here slice by slice); with rejection the kept rows are those
    whose foreground count (numpy) reaches keep_frac * a^2, offsets packed."""
    rng = np.random.default_rng(5)
    geom = synth.random_geometry(rng, n=8, n_stacks=2, W=30, H=26, K=3)
    offs, total = geom.stack_offsets()
    stacks = rng.uniform(0.0, 1.0, total).astype(np.float32)
    nk = sum(k for (_, _, k) in geom.stack_dims)
    sa = rng.choice([4, 6, 8, 12], nk).astype(np.int32)
    ss = (sa // 2).astype(np.int32)
    G = O.geom(geom)
    desc, npix = O.patches_build_sizes(G, stacks, sa, ss)
    rows, cnts, off, gk = [], [], 0, 0
    thr = np.float32(0.5) * stacks.max()
    for s, (W, H, K) in enumerate(geom.stack_dims):
        img = stacks[offs[s]:offs[s] + W * H * K].reshape(K, H, W)
        for k in range(K):
            a, st = int(sa[gk]), int(ss[gk])
            for y0 in range(0, H - a + 1, st):
                for x0 in range(0, W - a + 1, st):
                    rows.append([s, k, x0, y0, a, a, off, 0])
                    cnts.append(int((img[k, y0:y0 + a, x0:x0 + a] > thr).sum()))
                    off += a * a
            gk += 1
    rows = np.array(rows, dtype=np.int32)
    assert np.array_equal(desc, rows) and npix == off
    keep = np.array([c >= 0.5 * r[4] * r[5] for c, r in zip(cnts, rows)])
    kept = rows[keep].copy()
    kept[:, 6] = np.concatenate([[0], np.cumsum(kept[:-1, 4] * kept[:-1, 5])])
    desc2, npix2 = O.patches_build_sizes(G, stacks, sa, ss, fg_frac=0.5, keep_frac=0.5)
    assert 0 < desc2.shape[0] < rows.shape[0]
    assert np.array_equal(desc2, kept) and npix2 == int((kept[:, 4] * kept[:, 5]).sum())
    # uniform sizes reproduce the single-size builder
    d3, n3 = O.patches_build_sizes(G, stacks, np.full(nk, 8, np.int32), np.full(nk, 4, np.int32), 0.5, 0.5)
    d4, n4 = O.patches_build(G, stacks, 8, 4, 0.5, 0.5)
    assert np.array_equal(d3, d4) and n3 == n4


def test_taylor_sinc_psf_table():
    """kind 1: the in-plane weights are sinc(1.2067 d / FWHM) (numpy's sinc),
    half of the peak at d = FWHM / 2, the through-plane profile unchanged;
    the forward model still maps a constant volume to constant patches."""
    rng = np.random.default_rng(11)
    geom = synth.random_geometry(rng, n=12, n_stacks=2, W=10, H=9, K=3, pix=0.7)
    G = O.geom(geom)
    for fwhm in (1.2, 2.5):
        ps = O.psf(fwhm, 3, 2, 0.8, kind=1)
        gxy, gz = O.psf_table(G, ps, 0)
        d = np.arange(-3, 4)
        assert np.allclose(gxy, np.sinc(1.2067091288 * d / fwhm), rtol=1e-11, atol=1e-14)
        g0xy, g0z = O.psf_table(G, O.psf(fwhm, 3, 2, 0.8), 0)
        assert np.array_equal(gz, g0z)
    ps = O.psf(2.5, 3, 2, 0.8, kind=1)
    gh, _ = O.psf_table(G, O.psf(2.0, 1, 0, 0.8, kind=1), 0)
    assert abs(gh[2] - 0.5) < 1e-9          # half maximum one pixel out when FWHM = 2 px
    desc, npix = synth.all_patches(geom, 4, 3)
    poses = synth.random_poses(rng, desc.shape[0], rot=10.0, trans=1.0)
    fix = O.pose_fixed(G, ps, desc, poses)
    sim, valid, _ = O.simulate(G, ps, np.full(geom.n_vox, 7.0, np.float32), desc, fix, npix)
    assert valid.sum() > 0 and np.allclose(sim[valid == 1], 7.0, rtol=1e-12)


def test_samples_on_the_last_voxel_plane_read_that_plane():
    """A sample exactly on the upper boundary (index N-1) is inside and takes
    the value of that plane."""
    n = 16
    geom = _aligned_geometry(n)
    G = O.geom(geom)
    ps = O.psf(1.2, 0, 0, 1.0)
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1000, geom.n_vox).astype(np.float32)
    vol = x.reshape(n, n, n)
    # columns 10..15 shifted by +0 land on x = 10..15 (15 = N-1); slice 15 = z N-1;
    # rows 12..15 land on y = 12..15
    desc = np.array([[0, n - 1, 10, 12, 6, 4, 0, 0]], dtype=np.int32)
    fix = O.pose_fixed(G, ps, desc, np.zeros((1, 6)))
    sim, valid, _ = O.simulate(G, ps, x, desc, fix, 24)
    assert np.all(valid == 1)
    assert np.array_equal(sim, vol[n - 1, 12:16, 10:16].reshape(-1).astype(np.float64))


def test_skew_motion_workload():
    """Skew matrix of the adult-brain experiment; with theta = 0 the skewed
    slices equal the motion-free ones, with theta > 0 only odd slices move."""
    T = synth.skew_matrix(10.0)
    S = np.tan(np.radians(10.0))
    assert np.allclose(T, [[1, S, S], [S, 1, S], [S, S, 1]])
    c0 = synth.config_skew(theta_deg=0.0, n=24)
    c1 = synth.config_skew(theta_deg=8.0, n=24)
    for a, b in zip(c0["stacks"], c1["stacks"]):
        assert np.array_equal(a[0::2], b[0::2])
        assert np.abs(a[1::2] - b[1::2]).max() > 1.0
