// Per-patch kernels of the PVR hot path: forward model (K2), adjoint (K4)
// and NCC with pose gradient (K6a/K6b).
//
// Decomposition (Sec. III, patch-level and voxel-level parallelism, redone
// for sm_103a): one CTA per (patch, tile of at most T x T output pixels).
// The CTA first evaluates the through-plane PSF sum at every in-plane
// lattice point of its tile plus a kxy halo -- the lattice point (i, j)
// holds sum_zeta g_z(zeta) trilinear(x, q(i, j, zeta)) and sum_zeta g_z over
// in-volume samples -- into shared memory, then applies the separable
// in-plane Gaussian taps from shared memory.  Each trilinear sample is thus
// gathered once per tile instead of (2 kxy + 1)^2 times per pixel.  The
// adjoint runs the same steps transposed: per-pixel coefficients, the
// transposed in-plane taps into lattice weights, then a scatter of every
// in-volume sample into its 8 voxels.
//
// Sample positions are Q11.20 fixed point: q = o + i e_col + j e_row +
// zeta e_zeta in 32-bit two's-complement arithmetic (exact whenever the
// result is in range, which the pose kernel guarantees for the whole sample
// box), so in-volume tests and voxel indices are exact integers.
#include "pvr_internal.h"

namespace pvr {
namespace {

constexpr unsigned kFracMask = (1u << kFracBits) - 1u;

struct TileInfo {
    int p, t;                // patch, tile index
    int stack, w, h, off;    // patch
    int i0, j0, tw, th;      // tile pixel origin (patch-relative) and size
    int Lw, Lh, L;           // lattice of the tile incl. halo
    float rLw, rLh, rtw;     // 1 / Lw, 1 / Lh, 1 / tw for qdiv
    unsigned o[3], ei[3], ej[3], ez[3];
    bool ok;
};

// Integer quotient a / d for 0 <= a < 2^22 from r = 1 / d (float): the
// exact quotient (a + 0.5) / d lies at least 0.5 / d from an integer, and
// the two float roundings move it by at most (a + 0.5) / d * 2^-23 < 0.5 / d,
// so truncation gives floor(a / d).  Lattice and tile indices stay far
// below 2^22.
__device__ __forceinline__ int qdiv(int a, float r)
{
    return (int)(((float)a + 0.5f) * r);
}

// Pixel o (index into the patch-pixel arrays) belongs to its patch.
__device__ __forceinline__ bool member_ok(const Tiling &tl, size_t o)
{
    return !tl.member || tl.member[o];
}

// Tile slot processed at launch position k: with a patch launch order
// (Tiling::order) the patches' slots in that order, each patch's tiles
// together.  Results do not depend on the order: every tile writes its own
// partial sums.
__device__ __forceinline__ long long tile_at(const Tiling &tl, long long k)
{
    if (!tl.order) return k;
    const int q = (int)k / tl.tpp;   // slots < 2^31 (max_patches x tiles per patch)
    return (long long)__ldg(tl.order + q) * tl.tpp + ((int)k - q * tl.tpp);
}

// Decode block -> (patch, tile); returns false for an empty tile or a
// patch whose descriptor row failed validation in the pose kernel.
__device__ __forceinline__ bool tile_setup_at(long long gid, const int32_t *__restrict__ desc,
                                              const int32_t *__restrict__ fix, const Tiling &tl,
                                              int kxy, TileInfo &ti)
{
    ti.p = (int)(gid / tl.tpp);
    ti.t = (int)(gid % tl.tpp);
    const int32_t *d = desc + 8 * (size_t)ti.p;
    ti.stack = d[0];
    ti.w = d[4];
    ti.h = d[5];
    ti.off = d[6];
    int tx = ti.t % tl.tiles_x, ty = ti.t / tl.tiles_x;
    ti.i0 = tx * tl.T;
    ti.j0 = ty * tl.T;
    const int32_t *f = fix + kFixStride * (size_t)ti.p;
    ti.ok = f[12] != 0;
    // f[13] = 0: the descriptor row failed validation -- touch nothing
    if (f[13] == 0 || ti.i0 >= ti.w || ti.j0 >= ti.h) return false;
    ti.tw = min(tl.T, ti.w - ti.i0);
    ti.th = min(tl.T, ti.h - ti.j0);
    ti.Lw = ti.tw + 2 * kxy;
    ti.Lh = ti.th + 2 * kxy;
    ti.L = ti.Lw * ti.Lh;
    ti.rLw = 1.0f / (float)ti.Lw;
    ti.rLh = 1.0f / (float)ti.Lh;
    ti.rtw = 1.0f / (float)ti.tw;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        ti.o[r] = (unsigned)f[r];
        ti.ei[r] = (unsigned)f[3 + r];
        ti.ej[r] = (unsigned)f[6 + r];
        ti.ez[r] = (unsigned)f[9 + r];
    }
    return true;
}

struct VolDims {
    int nx, ny, nz;
    unsigned nxy;            // nx * ny (used where the volume has < 2^31 voxels)
    unsigned ux, uy, uz;     // (n - 1) << 20: largest in-volume coordinate
};

__host__ __device__ __forceinline__ VolDims vol_dims(int nx, int ny, int nz)
{
    VolDims v;
    v.nx = nx;
    v.ny = ny;
    v.nz = nz;
    v.nxy = (unsigned)nx * (unsigned)ny;
    v.ux = (unsigned)(nx - 1) << kFracBits;
    v.uy = (unsigned)(ny - 1) << kFracBits;
    v.uz = (unsigned)(nz - 1) << kFracBits;
    return v;
}

// Split an in-volume fixed-point coordinate into base voxel and fraction;
// the last plane is addressed as cell n-2 with fraction 1.
// FAST: the caller knows q < (n - 1) << 20, so no clamp is needed.
template <bool FAST = false>
__device__ __forceinline__ void split(unsigned q, int n, int &b, float &f)
{
    b = (int)(q >> kFracBits);
    // 1 + frac * 2^-20 has the fraction bits as its top mantissa bits, so
    // subtracting 1 gives (q & mask) * 2^-20 exactly (without a conversion)
    f = __uint_as_float(0x3f800000u | ((q & kFracMask) << (23 - kFracBits))) - 1.0f;
    if (!FAST && b == n - 1) {
        b = n - 2;
        f = 1.0f;
    }
}

// Traversal order of a tile's lattice, chosen per patch so that neighbouring
// lanes touch neighbouring voxels in memory (x fastest): lanes step along the
// patch columns, along the patch rows, or -- when the slice normal is the
// direction closest to the volume's x axis (e.g. sagittal slices) -- eight
// lanes share a lattice point, one per through-plane sample (needs
// 2 kz + 1 <= 8).  The order changes only the float32 summation order.
enum { kAlongCol = 0, kAlongRow = 1, kAlongZeta = 2 };

__device__ __forceinline__ float x_share(const unsigned e[3])
{
    float a = (float)(int)e[0], b = (float)(int)e[1], c = (float)(int)e[2];
    float n2 = a * a + b * b + c * c;
    return n2 > 0.f ? fabsf(a) * rsqrtf(n2) : 0.f;
}

__device__ __forceinline__ int pick_order(const TileInfo &ti, int kz)
{
    float ci = x_share(ti.ei), cj = x_share(ti.ej), cz = x_share(ti.ez);
    if (kz > 0 && 2 * kz + 1 <= 8 && cz > ci && cz > cj) return kAlongZeta;
    return cj > ci ? kAlongRow : kAlongCol;
}

// Tile-lattice coordinates (li, lj) (0-based, halo included) of item it.
__device__ __forceinline__ void lattice_coords(const TileInfo &ti, int order, int it, int &li, int &lj)
{
    if (order == kAlongRow) {
        li = qdiv(it, ti.rLh);
        lj = it - li * ti.Lh;
    } else {
        lj = qdiv(it, ti.rLw);
        li = it - lj * ti.Lw;
    }
}

// Fixed-point position of tile-lattice point (li, lj) at zeta = 0.
__device__ __forceinline__ void lattice_pos(const TileInfo &ti, int kxy, int li, int lj, unsigned q[3])
{
    int pi = ti.i0 - kxy + li, pj = ti.j0 - kxy + lj;
#pragma unroll
    for (int r = 0; r < 3; ++r) q[r] = ti.o[r] + (unsigned)pi * ti.ei[r] + (unsigned)pj * ti.ej[r];
}

// Volume sources of the gathers.  PlainVol reads the eight corners of a
// trilinear cell as eight 4-byte loads (any volume size).  QuadVol reads the
// quad copy of the volume, q[i] = (x[i], x[i + 1], x[i + nx], x[i + nx + 1])
// for voxel i, so a cell is two 16-byte loads (its two z planes); it needs
// fewer than 2^31 voxels.  Both give the same eight values.
struct PlainVol {
    const float *x;
};
struct QuadVol {
    const float4 *q;
};

__device__ __forceinline__ void cell_corners(const PlainVol &src, const VolDims &vd, int bx, int by,
                                             int bz, float v[8])
{
    const size_t nxy = (size_t)vd.nx * vd.ny;
    const float *b = src.x + (size_t)bz * nxy + (size_t)by * vd.nx + bx;
    v[0] = __ldg(b);
    v[1] = __ldg(b + 1);
    v[2] = __ldg(b + vd.nx);
    v[3] = __ldg(b + vd.nx + 1);
    v[4] = __ldg(b + nxy);
    v[5] = __ldg(b + nxy + 1);
    v[6] = __ldg(b + nxy + vd.nx);
    v[7] = __ldg(b + nxy + vd.nx + 1);
}

__device__ __forceinline__ void cell_corners(const QuadVol &src, const VolDims &vd, int bx, int by,
                                             int bz, float v[8])
{
    const unsigned i = ((unsigned)bz * (unsigned)vd.ny + (unsigned)by) * (unsigned)vd.nx + (unsigned)bx;
    const float4 lo = __ldg(src.q + i), hi = __ldg(src.q + i + vd.nxy);
    v[0] = lo.x;
    v[1] = lo.y;
    v[2] = lo.z;
    v[3] = lo.w;
    v[4] = hi.x;
    v[5] = hi.y;
    v[6] = hi.z;
    v[7] = hi.w;
}

// Trilinear value at a fixed-point position inside the volume; corners v
// ordered (x, y, z) = 000, 100, 010, 110, 001, 101, 011, 111.
template <bool FAST = false, class SRC>
__device__ __forceinline__ float trilinear(const SRC &src, const VolDims &vd, unsigned qx, unsigned qy,
                                           unsigned qz)
{
    int bx, by, bz;
    float fx, fy, fz;
    split<FAST>(qx, vd.nx, bx, fx);
    split<FAST>(qy, vd.ny, by, fy);
    split<FAST>(qz, vd.nz, bz, fz);
    float v[8];
    cell_corners(src, vd, bx, by, bz, v);
    float c00 = fmaf(fx, v[1] - v[0], v[0]);
    float c10 = fmaf(fx, v[3] - v[2], v[2]);
    float c01 = fmaf(fx, v[5] - v[4], v[4]);
    float c11 = fmaf(fx, v[7] - v[6], v[6]);
    float c0 = fmaf(fy, c10 - c00, c00);
    float c1 = fmaf(fy, c11 - c01, c01);
    return fmaf(fz, c1 - c0, c0);
}

__device__ __forceinline__ bool inside(const VolDims &vd, unsigned qx, unsigned qy, unsigned qz)
{
    return qx <= vd.ux && qy <= vd.uy && qz <= vd.uz;
}

// True when every sample of the tile (lattice with halo, every zeta) lies
// strictly inside the volume, so that loops need no in-volume test and no
// last-plane clamp.  Sample positions are affine in (column, row, zeta): the
// extremes sit at the 8 corners of the sample box.
__device__ __forceinline__ bool tile_interior(const TileInfo &ti, const VolDims &vd, int kxy, int kz)
{
    if (!ti.ok) return false;
    const unsigned lim[3] = {vd.ux, vd.uy, vd.uz};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        int pi = ti.i0 - kxy + ((c & 1) ? ti.Lw - 1 : 0);
        int pj = ti.j0 - kxy + ((c & 2) ? ti.Lh - 1 : 0);
        int z = (c & 4) ? kz : -kz;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            unsigned q = ti.o[r] + (unsigned)pi * ti.ei[r] + (unsigned)pj * ti.ej[r] + (unsigned)z * ti.ez[r];
            if (q >= lim[r]) return false;
        }
    }
    return true;
}

// True when every through-plane sample of the lattice point at q0 lies
// strictly inside the volume (the FAST condition of tile_interior for one
// walk): positions are affine in zeta, so its two end samples decide.  Used
// in border tiles to run the lanes whose walks are inside on the FAST code
// (same results: the in-volume tests pass and no clamp applies).
__device__ __forceinline__ bool walk_inside(const VolDims &vd, const TileInfo &ti, const unsigned q0[3], int kz)
{
    const unsigned lim[3] = {vd.ux, vd.uy, vd.uz};
    bool ok = true;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const unsigned a = q0[r] - (unsigned)kz * ti.ez[r], b = q0[r] + (unsigned)kz * ti.ez[r];
        ok = ok && a < lim[r] && b < lim[r];
    }
    return ok;
}

// Through-plane walks with cell-face reuse.  The through-plane samples of a
// lattice point are one PSF step apart along e_zeta.  Walking them in the
// direction in which e_zeta's largest voxel component FA is positive, a
// sample whose cell starts one voxel further along FA (and in the same cell
// along the two other axes) shares its lower face with the previous
// sample's upper face: the adjoint merges the two contributions to those 4
// voxels before one set of reductions.  The test compares exact voxel
// indices, so it only removes duplicate memory operations.
struct Walk {
    int fa, z0, dz;
};

__device__ __forceinline__ Walk zeta_walk(const TileInfo &ti, int kz)
{
    int c0 = abs((int)ti.ez[0]), c1 = abs((int)ti.ez[1]), c2 = abs((int)ti.ez[2]);
    Walk w;
    w.fa = (c2 >= c1 && c2 >= c0) ? 2 : (c1 >= c0 ? 1 : 0);
    const bool up = (int)ti.ez[w.fa] >= 0;
    w.dz = up ? 1 : -1;
    w.z0 = up ? -kz : kz;
    return w;
}

template <int FA>
struct FaceAxes;
template <>
struct FaceAxes<0> {
    static constexpr int A1 = 1, A2 = 2;
};
template <>
struct FaceAxes<1> {
    static constexpr int A1 = 0, A2 = 2;
};
template <>
struct FaceAxes<2> {
    static constexpr int A1 = 0, A2 = 1;
};

__device__ __forceinline__ size_t axis_stride(const VolDims &vd, int a)
{
    return a == 0 ? (size_t)1 : (a == 1 ? (size_t)vd.nx : (size_t)vd.nx * vd.ny);
}

// One cell face from every lane of a warp (valid lanes only), merged across
// neighbouring lanes first.  Lanes hold neighbouring lattice points along the
// traversal axis, so lane l + 1's face usually starts one voxel further along
// A1 than lane l's: then its two low-A1 corners are lane l's two high-A1
// corners, lane l adds them to its own before reducing, and lane l + 1 skips
// them.  The test compares exact voxel indices (a volume of fewer than 2^31
// voxels, interior cells only, so index + s1 never wraps), so it only removes
// duplicate reductions: about a quarter of them per face.  Every lane of the
// warp must call this together.
template <bool PAIR>
__device__ __forceinline__ void face_red_warp(float *addon, float *conf, bool valid, unsigned idx,
                                              unsigned s1, unsigned s2, float r[4], float w[4])
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned key = valid ? idx : 0xffffffffu;
    const unsigned nkey = __shfl_down_sync(full, key, 1);
    const float nr0 = __shfl_down_sync(full, r[0], 1), nr2 = __shfl_down_sync(full, r[2], 1);
    const float nw0 = __shfl_down_sync(full, w[0], 1), nw2 = __shfl_down_sync(full, w[2], 1);
    const bool take = valid && lane != 31 && nkey == key + s1;
    if (take) {
        r[1] += nr0;
        r[3] += nr2;
        w[1] += nw0;
        w[3] += nw2;
    }
    const bool given = __shfl_up_sync(full, take, 1) && lane != 0;
    if (!valid) return;
    auto red = [&](unsigned i, float a, float b) {
        if (PAIR) {
            atomicAdd(reinterpret_cast<float2 *>(addon) + i, make_float2(a, b));
        } else {
            if (addon) atomicAdd(addon + i, a);
            if (conf) atomicAdd(conf + i, b);
        }
    };
    if (!given) {
        red(idx, r[0], w[0]);
        red(idx + s2, r[2], w[2]);
    }
    red(idx + s1, r[1], w[1]);
    red(idx + s1 + s2, r[3], w[3]);
}

// walk_scatter with the faces merged across lanes (face_red_warp): every
// lane of the warp runs the same walk; lanes without a lattice point (act
// false) and samples outside the volume take part with no reductions of
// their own.  FAST: interior tile (no in-volume tests, no last-plane clamp).
template <int FA, int KZ, bool PAIR, bool FAST>
__device__ __forceinline__ void walk_scatter_warp(const VolDims &vd, const TileInfo &ti, const unsigned q0[3],
                                                  int kz_rt, const float *__restrict__ gz, const Walk &wk,
                                                  float ur, float uw, bool act, float *addon, float *conf)
{
    constexpr int A1 = FaceAxes<FA>::A1, A2 = FaceAxes<FA>::A2;
    const unsigned full = 0xffffffffu;
    const int kz = KZ >= 0 ? KZ : kz_rt;
    const unsigned s1 = (unsigned)axis_stride(vd, A1), s2 = (unsigned)axis_stride(vd, A2);
    const unsigned sf = (unsigned)axis_stride(vd, FA);
    float pr[4] = {0.f, 0.f, 0.f, 0.f}, pw[4] = {0.f, 0.f, 0.f, 0.f};
    unsigned pidx = 0;
    bool have = false;
    int pb[3] = {-2, -2, -2};
#pragma unroll 1
    for (int t = 0; t <= 2 * kz; ++t) {
        const int z = wk.z0 + t * wk.dz;
        const unsigned qx = q0[0] + (unsigned)z * ti.ez[0], qy = q0[1] + (unsigned)z * ti.ez[1];
        const unsigned qz = q0[2] + (unsigned)z * ti.ez[2];
        const bool ins = FAST || inside(vd, qx, qy, qz);
        int b[3];
        float f[3];
        split<FAST>(qx, vd.nx, b[0], f[0]);
        split<FAST>(qy, vd.ny, b[1], f[1]);
        split<FAST>(qz, vd.nz, b[2], f[2]);
        const unsigned idx = ((unsigned)b[2] * (unsigned)vd.ny + (unsigned)b[1]) * (unsigned)vd.nx + (unsigned)b[0];
        const float g = gz[z + kz];
        const float f1 = f[A1], f2 = f[A2];
        const float wf[4] = {(1.f - f1) * (1.f - f2), f1 * (1.f - f2), (1.f - f1) * f2, f1 * f2};
        const float ar = g * ur, aw = g * uw;
        const float lo = 1.f - f[FA], hi = f[FA];
        float lr[4], lw[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            lr[k] = ar * lo * wf[k];
            lw[k] = aw * lo * wf[k];
        }
        // the previous sample's upper face: merged into this lower face when
        // it is the same face, else reduced on its own
        const bool merge = have && ins && b[FA] == pb[FA] + 1 && b[A1] == pb[A1] && b[A2] == pb[A2];
        const bool pv = act && have && !merge;
        if (__any_sync(full, pv)) face_red_warp<PAIR>(addon, conf, pv, pidx, s1, s2, pr, pw);
        if (merge) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                lr[k] += pr[k];
                lw[k] += pw[k];
            }
        }
        const bool cv = act && ins;
        if (FAST || __any_sync(full, cv)) face_red_warp<PAIR>(addon, conf, cv, idx, s1, s2, lr, lw);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            pr[k] = ar * hi * wf[k];
            pw[k] = aw * hi * wf[k];
        }
        pidx = idx + sf;
        have = ins;
        pb[0] = b[0];
        pb[1] = b[1];
        pb[2] = b[2];
    }
    const bool pv = act && have;
    if (__any_sync(full, pv)) face_red_warp<PAIR>(addon, conf, pv, pidx, s1, s2, pr, pw);
}

// Through-plane PSF sums of one lattice point: acc = sum g_z trilinear
// (when want_a), den = sum g_z over the in-volume samples.
template <int KZ, bool FAST, class SRC>
__device__ __forceinline__ void walk_forward(const SRC &src, const VolDims &vd, const TileInfo &ti,
                                             const unsigned q0[3], int kz_rt, const float *__restrict__ gz,
                                             bool want_a, float &acc, float &den)
{
    const int kz = KZ >= 0 ? KZ : kz_rt;
#pragma unroll
    for (int z = -kz; z <= kz; ++z) {
        unsigned qx = q0[0] + (unsigned)z * ti.ez[0];
        unsigned qy = q0[1] + (unsigned)z * ti.ez[1];
        unsigned qz = q0[2] + (unsigned)z * ti.ez[2];
        if (FAST || inside(vd, qx, qy, qz)) {
            float g = gz[z + kz];
            if (want_a) acc = fmaf(g, trilinear<FAST>(src, vd, qx, qy, qz), acc);
            den += g;
        }
    }
}

// Phase 1 of the forward model: through-plane PSF sums at every lattice
// point of the tile (stored row-major).  A (may be null) <- sum g_z
// trilinear, B <- sum g_z over in-volume samples.
template <int KZ, bool FAST = false, class SRC = PlainVol>
__device__ __forceinline__ void lattice_forward(const SRC src, const VolDims &vd,
                                                const TileInfo &ti, int kxy, int kz_rt,
                                                const float *__restrict__ gz, int order, float *A,
                                                float *B)
{
    const int kz = KZ >= 0 ? KZ : kz_rt;
    if (order != kAlongZeta) {
        for (int it = threadIdx.x; it < ti.L; it += blockDim.x) {
            int li, lj;
            lattice_coords(ti, order, it, li, lj);
            unsigned q0[3];
            lattice_pos(ti, kxy, li, lj, q0);
            float acc = 0.f, den = 0.f;
            // border tile: warps whose walks are all inside take the FAST code
            if (FAST || __all_sync(__activemask(), walk_inside(vd, ti, q0, kz)))
                walk_forward<KZ, true>(src, vd, ti, q0, kz, gz, A != nullptr, acc, den);
            else
                walk_forward<KZ, false>(src, vd, ti, q0, kz, gz, A != nullptr, acc, den);
            int sidx = lj * ti.Lw + li;
            if (A) A[sidx] = acc;
            B[sidx] = den;
        }
        return;
    }
    const int zl = threadIdx.x & 7;
    const bool zon = zl <= 2 * kz;
    const int zeta = zl - kz;
    const float g = zon ? gz[zl] : 0.f;
    const int ngrp = blockDim.x >> 3;
    for (int base = 0; base < ti.L; base += ngrp) {
        int lp = base + (threadIdx.x >> 3);
        float a = 0.f, b = 0.f;
        if (zon && lp < ti.L) {
            unsigned q[3];
            const int lj = qdiv(lp, ti.rLw);
                lattice_pos(ti, kxy, lp - lj * ti.Lw, lj, q);
            unsigned qx = q[0] + (unsigned)zeta * ti.ez[0];
            unsigned qy = q[1] + (unsigned)zeta * ti.ez[1];
            unsigned qz = q[2] + (unsigned)zeta * ti.ez[2];
            if (FAST || inside(vd, qx, qy, qz)) {
                if (A) a = g * trilinear<FAST>(src, vd, qx, qy, qz);
                b = g;
            }
        }
        // reduce-scatter over the group of 8: lanes 0-3 end with sum a,
        // lanes 4-7 with sum b
        const bool hi4 = zl & 4;
        float t = (hi4 ? b : a) + __shfl_xor_sync(0xffffffffu, hi4 ? a : b, 4);
        t += __shfl_xor_sync(0xffffffffu, t, 2);
        t += __shfl_xor_sync(0xffffffffu, t, 1);
        if (lp < ti.L) {
            if (zl == 0 && A) A[lp] = t;
            if (zl == 4) B[lp] = t;
        }
    }
}

// In-plane taps at tile pixel (ci, cj) from lattice array V.
__device__ __forceinline__ float inplane(const float *V, int Lw, int kxy, const float *gxy, int ci,
                                         int cj)
{
    float s = 0.f;
    for (int dj = -kxy; dj <= kxy; ++dj) {
        const float *row = V + (cj + kxy + dj) * Lw + ci + kxy;
        float r = 0.f;
        for (int di = -kxy; di <= kxy; ++di) r = fmaf(gxy[di + kxy], row[di], r);
        s = fmaf(gxy[dj + kxy], r, s);
    }
    return s;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sums of NV doubles (block size multiple of 32, <= 1024);
// result valid in thread 0.  red: shared scratch of 32 * NV doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double *v, double *red)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < NV; ++k) red[wid * NV + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += red[w * NV + k];
            v[k] = s;
        }
    __syncthreads();
}

// Block-wide float32 sums of NV values; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum_f(float *v, float *red)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < NV; ++k) red[wid * NV + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < NV; ++k) {
            float s = 0.f;
            for (int w = 0; w < nw; ++w) s += red[w * NV + k];
            v[k] = s;
        }
    __syncthreads();
}

// Float-float accumulator: an unevaluated sum hi + lo of float32s, updated
// with error-free transformations (two-sum; exact products by fma), so sums
// of products keep about 44 bits -- enough for variances computed as
// differences of raw moments, at float32 speed.
struct FFSum {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float a)
    {
        float s = hi + a;
        float bb = s - hi;
        float err = (hi - (s - bb)) + (a - bb);
        hi = s;
        lo += err;
    }
    __device__ __forceinline__ void add_prod(float a, float b)
    {
        float p = a * b;
        float e = fmaf(a, b, -p);
        add(p);
        lo += e;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Warp sum of float-float values (two-sum at every level, about 48
// significant bits) on the float32 pipe: float64 arithmetic runs at a small
// fraction of the float32 rate on this GPU, so per-thread double shuffles and
// adds would dominate a tile's reductions.
__device__ __forceinline__ void warp_sum_ff(float &hi, float &lo)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
        const float s = hi + oh, bb = s - hi;
        const float err = (hi - (s - bb)) + (oh - bb);
        hi = s;
        lo = (lo + ol) + err;
    }
}

// Block sums of NV float-float accumulators as doubles in out (valid in
// thread 0): float-float within each warp, float64 across the warps.
// red: shared scratch of 32 * NV doubles.  Ends with a barrier.  Not
// inlined (see block_sum_fd).
template <int NV>
__device__ __noinline__ void block_sum_ff(FFSum (&f)[NV], double (&out)[NV], double *red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) warp_sum_ff(f[k].hi, f[k].lo);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[wid * NV + k] = f[k].value();
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += red[w * NV + k];
            out[k] = t;
        }
    __syncthreads();
}

// Block sums of NV float32 values as doubles in out (valid in thread 0):
// float32 within each warp (32 terms), float64 across the warps.  Ends with
// a barrier.  Not inlined: inlined into the persistent kernels it made the
// register allocator spill hundreds of bytes of their tile loops.
template <int NV>
__device__ __noinline__ void block_sum_fd(float (&v)[NV], double (&out)[NV], double *red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[wid * NV + k] = (double)v[k];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += red[w * NV + k];
            out[k] = t;
        }
    __syncthreads();
}

// ------------------------------------------------------------------ K2 --
// Forward model.  y == null: write sim, valid.  y != null: write the
// residual e = y - sim (0 where invalid) and valid, plus per-tile partials
// {N_valid, sum e^2, min e, max e} for the EM step.
// One (patch, tile) slot gid of the forward model; sm: dynamic shared memory.
// Ends with every thread past its last shared-memory read.
template <int KXY, int KZ, class SRC>
__device__ __forceinline__ void simulate_tile(long long gid, const SRC &x, const VolDims &vd,
                                              const int32_t *__restrict__ desc,
                                              const int32_t *__restrict__ fix, const PsfTab &psf,
                                              const Tiling &tl, const float *__restrict__ y,
                                              float *__restrict__ out, uint8_t *__restrict__ valid,
                                              double *__restrict__ part, float *sm)
{
    __shared__ float fred[32 * 2];
    const int kxy = KXY >= 0 ? KXY : psf.kxy;
    TileInfo ti;
    bool has = tile_setup_at(gid, desc, fix, tl, kxy, ti);
    if (!has) {
        if (part && threadIdx.x < kPartStride)
            part[(size_t)gid * kPartStride + threadIdx.x] = 0.0;
        return;
    }
    float *A = sm, *B = sm + ti.L;
    if (ti.ok) {
        const int kz = KZ >= 0 ? KZ : psf.kz;
        const int order = pick_order(ti, kz);
        if (tile_interior(ti, vd, kxy, kz))
            lattice_forward<KZ, true, SRC>(x, vd, ti, kxy, kz, psf.gz[ti.stack], order, A, B);
        else
            lattice_forward<KZ, false, SRC>(x, vd, ti, kxy, kz, psf.gz[ti.stack], order, A, B);
    } else {
        for (int lp = threadIdx.x; lp < ti.L; lp += blockDim.x) A[lp] = B[lp] = 0.f;
    }
    __syncthreads();
    float se2 = 0.f, emin = INFINITY, emax = -INFINITY;
    int nval = 0;
    const int np = ti.tw * ti.th;
    for (int pp = threadIdx.x; pp < np; pp += blockDim.x) {
        const int cj = qdiv(pp, ti.rtw), ci = pp - cj * ti.tw;
        float num = inplane(A, ti.Lw, kxy, psf.gxy, ci, cj);
        float den = inplane(B, ti.Lw, kxy, psf.gxy, ci, cj);
        size_t o = (size_t)ti.off + (size_t)(ti.j0 + cj) * ti.w + (ti.i0 + ci);
        bool v = den > 0.f && member_ok(tl, o);
        float s = v ? num / den : 0.f;
        if (y) {
            float e = v ? __ldg(y + o) - s : 0.f;
            out[o] = e;
            if (v) {
                se2 = fmaf(e, e, se2);
                emin = fminf(emin, e);
                emax = fmaxf(emax, e);
                ++nval;
            }
        } else {
            out[o] = s;
        }
        valid[o] = v ? 1 : 0;
    }
    if (part) {
        float acc[2] = {(float)nval, se2};
        float mn = warp_min(emin), mx = warp_max(emax);
        __shared__ float rmn[32], rmx[32];
        int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) {
            rmn[wid] = mn;
            rmx[wid] = mx;
        }
        block_sum_f<2>(acc, fred);
        if (threadIdx.x == 0) {
            float a = INFINITY, b = -INFINITY;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                a = fminf(a, rmn[w]);
                b = fmaxf(b, rmx[w]);
            }
            double *pt = part + (size_t)gid * kPartStride;
            pt[0] = (double)acc[0];
            pt[1] = (double)acc[1];
            pt[2] = (double)a;
            pt[3] = (double)b;
        }
    } else {
        __syncthreads();
    }
}

// Forward model, one CTA per (patch, tile) slot.
template <int KXY, int KZ, class SRC>
__global__ void __launch_bounds__(256) k_simulate(const SRC x, VolDims vd,
                                                  const int32_t *__restrict__ desc,
                                                  const int32_t *__restrict__ fix, PsfTab psf,
                                                  Tiling tl, const float *__restrict__ y,
                                                  float *__restrict__ out,
                                                  uint8_t *__restrict__ valid,
                                                  double *__restrict__ part)
{
    extern __shared__ float sm[];
    simulate_tile<KXY, KZ, SRC>(tile_at(tl, blockIdx.x), x, vd, desc, fix, psf, tl, y, out, valid, part, sm);
}

// Next work item of a persistent CTA from the queue counter (thread 0 takes
// it, the block reads it after the barrier); >= n_items: queue empty.
__device__ __forceinline__ int next_item(int *counter, int *slot)
{
    if (threadIdx.x == 0) *slot = atomicAdd(counter, 1);
    __syncthreads();
    return *slot;
}

// Forward model as a persistent work queue over the non-empty (patch, tile)
// slots listed in items (largest tiles first): one launch serves patches of
// every size, and CTAs that finish early take more tiles.
template <int KXY, int KZ, class SRC>
__global__ void __launch_bounds__(256) k_simulate_q(const SRC x, VolDims vd,
                                                    const int32_t *__restrict__ desc,
                                                    const int32_t *__restrict__ fix, PsfTab psf,
                                                    Tiling tl, const float *__restrict__ y,
                                                    float *__restrict__ out,
                                                    uint8_t *__restrict__ valid,
                                                    double *__restrict__ part,
                                                    const int32_t *__restrict__ items, int n_items,
                                                    int *counter)
{
    extern __shared__ float sm[];
    __shared__ int cur;
    for (;;) {
        const int it = next_item(counter, &cur);
        if (it >= n_items) break;
        simulate_tile<KXY, KZ, SRC>(items[it], x, vd, desc, fix, psf, tl, y, out, valid, part, sm);
        __syncthreads();
    }
}

// Pixel coefficients (of the adjoint and of the NCC gradient) live in a
// zero-padded array:
// pixel (ci, cj) of the tile at Cp[(cj + 2 kxy) cw + ci + 2 kxy] with
// cw = tw + 4 kxy, so that the transposed in-plane taps of every lattice
// point (halo included) read in bounds without tests.  At most
// (T + 4 kxy)^2 floats.
__device__ __forceinline__ int cpad_w(const TileInfo &ti, int kxy) { return ti.tw + 4 * kxy; }
__device__ __forceinline__ int cpad_at(const TileInfo &ti, int kxy, int ci, int cj)
{
    return (cj + 2 * kxy) * cpad_w(ti, kxy) + ci + 2 * kxy;
}

// Zero the border of the padded coefficient array (the pixels' entries are
// written by the pixel loops).
__device__ __forceinline__ void cpad_border(const TileInfo &ti, int kxy, float *Cp)
{
    const int cw = cpad_w(ti, kxy), b = 2 * kxy, top = 2 * b * cw, side = 2 * b * ti.th;
    for (int k = threadIdx.x; k < top + side; k += blockDim.x) {
        int at;
        if (k < top) {
            const int r = k / cw, c = k - r * cw;                // rows 0..b-1, then the b below the tile
            at = (r < b ? r : ti.th + r) * cw + c;
        } else {
            const int t = k - top, r = t / (2 * b), c = t - r * 2 * b;   // b columns each side
            at = (r + b) * cw + (c < b ? c : ti.tw + c);
        }
        Cp[at] = 0.f;
    }
}

// ------------------------------------------------------------------ K4 --
// Adjoint.  Pixel coefficients cr = w r / den, cw = w / den (valid pixels),
// transposed in-plane taps into lattice weights U, U', then every in-volume
// sample adds U g_z tri and U' g_z tri to its 8 voxels (float atomics;
// PAIR = interleaved (addon, conf) float2 pairs with one vector reduction
// per voxel, otherwise two separate arrays).

// Phase 3 of the adjoint: scatter of every in-volume sample of the tile in
// its traversal order (FAST: interior tile, no in-volume tests).
template <int KZ, bool PAIR, bool FAST>
__device__ __forceinline__ void adjoint_scatter(const VolDims &vd, const TileInfo &ti, int kxy, int kz,
                                                const float *__restrict__ gz, const float *U,
                                                const float *Uw, float *addon, float *conf)
{
    const int order = pick_order(ti, kz);
    if (order != kAlongZeta) {
        // warps walk together and merge faces across lanes
        const Walk wk = zeta_walk(ti, kz);
        for (int base = threadIdx.x & ~31; base < ti.L; base += blockDim.x) {
            const int it = base + (threadIdx.x & 31);
            bool act = false;
            float ur = 0.f, uw = 0.f;
            unsigned q0[3] = {0u, 0u, 0u};
            if (it < ti.L) {
                int li, lj;
                lattice_coords(ti, order, it, li, lj);
                const int sidx = lj * ti.Lw + li;
                ur = U[sidx];
                uw = Uw[sidx];
                act = ur != 0.f || uw != 0.f;
                lattice_pos(ti, kxy, li, lj, q0);
            }
            if (!__any_sync(0xffffffffu, act)) continue;
            // border tile: warps whose walks are all inside take the FAST code
            if (FAST || __all_sync(0xffffffffu, !act || walk_inside(vd, ti, q0, kz))) {
                if (wk.fa == 2) walk_scatter_warp<2, KZ, PAIR, true>(vd, ti, q0, kz, gz, wk, ur, uw, act, addon, conf);
                else if (wk.fa == 1) walk_scatter_warp<1, KZ, PAIR, true>(vd, ti, q0, kz, gz, wk, ur, uw, act, addon, conf);
                else walk_scatter_warp<0, KZ, PAIR, true>(vd, ti, q0, kz, gz, wk, ur, uw, act, addon, conf);
            } else {
                if (wk.fa == 2) walk_scatter_warp<2, KZ, PAIR, false>(vd, ti, q0, kz, gz, wk, ur, uw, act, addon, conf);
                else if (wk.fa == 1) walk_scatter_warp<1, KZ, PAIR, false>(vd, ti, q0, kz, gz, wk, ur, uw, act, addon, conf);
                else walk_scatter_warp<0, KZ, PAIR, false>(vd, ti, q0, kz, gz, wk, ur, uw, act, addon, conf);
            }
        }
    } else {
        // eight lanes per lattice point, one per through-plane sample; the
        // samples step mostly along x here, so lane zl + 1's cell usually
        // starts one voxel after lane zl's: its four low-x corners are lane
        // zl's four high-x corners, added there before the reductions
        // (exact index comparison, as in face_red_warp)
        const unsigned full = 0xffffffffu;
        const int zl = threadIdx.x & 7, zeta = zl - kz;
        const bool zon = zl <= 2 * kz;
        const float g = zon ? gz[zl] : 0.f;
        const int ngrp = blockDim.x >> 3;
        const unsigned nx = (unsigned)vd.nx, nxy = vd.nxy;
        for (int base = 0; base < ti.L; base += ngrp) {
            const int lp = base + (threadIdx.x >> 3);
            bool valid = false;
            unsigned idx = 0xffffffffu;
            float cr[2][2][2], cw[2][2][2];   // [z][y][x] corner contributions
            if (zon && lp < ti.L) {
                const float ur = U[lp], uw = Uw[lp];
                unsigned q[3];
                const int lj = qdiv(lp, ti.rLw);
                lattice_pos(ti, kxy, lp - lj * ti.Lw, lj, q);
                const unsigned qx = q[0] + (unsigned)zeta * ti.ez[0];
                const unsigned qy = q[1] + (unsigned)zeta * ti.ez[1];
                const unsigned qz = q[2] + (unsigned)zeta * ti.ez[2];
                valid = (ur != 0.f || uw != 0.f) && (FAST || inside(vd, qx, qy, qz));
                if (valid) {
                    int bx, by, bz;
                    float fx, fy, fz;
                    split<FAST>(qx, vd.nx, bx, fx);
                    split<FAST>(qy, vd.ny, by, fy);
                    split<FAST>(qz, vd.nz, bz, fz);
                    idx = ((unsigned)bz * (unsigned)vd.ny + (unsigned)by) * nx + (unsigned)bx;
                    const float wx[2] = {1.f - fx, fx}, wy[2] = {1.f - fy, fy}, wz[2] = {1.f - fz, fz};
                    const float ar = g * ur, aw = g * uw;
#pragma unroll
                    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
                        for (int cy = 0; cy < 2; ++cy)
#pragma unroll
                            for (int cx = 0; cx < 2; ++cx) {
                                const float t = wx[cx] * wy[cy] * wz[cz];
                                cr[cz][cy][cx] = ar * t;
                                cw[cz][cy][cx] = aw * t;
                            }
                }
            }
            if (!__any_sync(full, valid)) continue;
            if (!valid) {
#pragma unroll
                for (int c = 0; c < 4; ++c) cr[c >> 1][c & 1][0] = cw[c >> 1][c & 1][0] = 0.f;
            }
            const unsigned nkey = __shfl_down_sync(full, idx, 1, 8);
            float nr[4], nw[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                nr[c] = __shfl_down_sync(full, cr[c >> 1][c & 1][0], 1, 8);
                nw[c] = __shfl_down_sync(full, cw[c >> 1][c & 1][0], 1, 8);
            }
            const bool take = valid && zl < 7 && nkey == idx + 1u;
            if (take) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    cr[c >> 1][c & 1][1] += nr[c];
                    cw[c >> 1][c & 1][1] += nw[c];
                }
            }
            const bool given = __shfl_up_sync(full, take, 1, 8) && zl > 0;
            if (!valid) continue;
#pragma unroll
            for (int cz = 0; cz < 2; ++cz)
#pragma unroll
                for (int cy = 0; cy < 2; ++cy)
#pragma unroll
                    for (int cx = 0; cx < 2; ++cx) {
                        if (cx == 0 && given) continue;
                        const unsigned at = idx + (unsigned)cz * nxy + (unsigned)cy * nx + (unsigned)cx;
                        if (PAIR) {
                            atomicAdd(reinterpret_cast<float2 *>(addon) + at,
                                      make_float2(cr[cz][cy][cx], cw[cz][cy][cx]));
                        } else {
                            if (addon) atomicAdd(addon + at, cr[cz][cy][cx]);
                            if (conf) atomicAdd(conf + at, cw[cz][cy][cx]);
                        }
                    }
        }
    }
}

// One (patch, tile) slot gid of the adjoint; sm: dynamic shared memory.
template <int KXY, int KZ, bool PAIR>
__device__ __forceinline__ void adjoint_tile(long long gid, const VolDims &vd,
                                             const int32_t *__restrict__ desc,
                                             const int32_t *__restrict__ fix, const PsfTab &psf,
                                             const Tiling &tl, const float *__restrict__ r,
                                             const float *__restrict__ w,
                                             const uint8_t *__restrict__ pmask,
                                             const float *__restrict__ pweight,
                                             float *__restrict__ addon, float *__restrict__ conf,
                                             float *sm)
{
    const int kxy = KXY >= 0 ? KXY : psf.kxy;
    const int kz = KZ >= 0 ? KZ : psf.kz;
    TileInfo ti;
    if (!tile_setup_at(gid, desc, fix, tl, kxy, ti) || !ti.ok) return;
    if (pmask && pmask[ti.p] == 0) return;
    const float pw = pweight ? pweight[ti.p] : 1.f;   // per-patch factor on r only
    const int np = ti.tw * ti.th;
    // pixel coefficients in zero-padded arrays (cpad_at): the transposed taps
    // of phase 2 then read in bounds without tests
    const int cw_ = cpad_w(ti, kxy);
    float *U = sm, *Uw = sm + ti.L, *CR = sm + 2 * ti.L, *CW = CR + cw_ * (ti.th + 4 * kxy);
    const float *gz = psf.gz[ti.stack];
    const bool interior = tile_interior(ti, vd, kxy, kz);
    // phase 0: in-volume PSF weight per lattice point (no gathers); inside
    // the volume every sample counts
    if (interior) {
        float b = 0.f;
        for (int z = -kz; z <= kz; ++z) b += gz[z + kz];
        for (int lp = threadIdx.x; lp < ti.L; lp += blockDim.x) U[lp] = b;
    } else {
        lattice_forward<KZ>(PlainVol{nullptr}, vd, ti, kxy, kz, gz, kAlongCol, nullptr, U);
    }
    __syncthreads();
    // phase 1: pixel coefficients
    cpad_border(ti, kxy, CR);
    cpad_border(ti, kxy, CW);
    for (int pp = threadIdx.x; pp < np; pp += blockDim.x) {
        const int cj = qdiv(pp, ti.rtw), ci = pp - cj * ti.tw;
        float den = inplane(U, ti.Lw, kxy, psf.gxy, ci, cj);
        size_t o = (size_t)ti.off + (size_t)(ti.j0 + cj) * ti.w + (ti.i0 + ci);
        float cr = 0.f, cw = 0.f;
        if (den > 0.f && member_ok(tl, o)) {
            float ww = w ? __ldg(w + o) : 1.f;
            float rr = r ? __ldg(r + o) : 1.f;
            cw = ww / den;
            cr = cw * rr;
            if (pweight) cr *= pw;
        }
        CR[cpad_at(ti, kxy, ci, cj)] = cr;
        CW[cpad_at(ti, kxy, ci, cj)] = cw;
    }
    __syncthreads();
    // phase 2: transposed in-plane taps into lattice weights
    for (int lp = threadIdx.x; lp < ti.L; lp += blockDim.x) {
        const int lj = qdiv(lp, ti.rLw), li = lp - lj * ti.Lw;   // lattice point = pixel (li - kxy, lj - kxy) of the tile
        const int at = (lj + kxy) * cw_ + (li + kxy);          // that pixel in the padded arrays
        float ur = 0.f, uw = 0.f;
#pragma unroll
        for (int dj = -kxy; dj <= kxy; ++dj) {
            float rr = 0.f, rw = 0.f;
#pragma unroll
            for (int di = -kxy; di <= kxy; ++di) {
                const float g = psf.gxy[di + kxy];
                rr = fmaf(g, CR[at - dj * cw_ - di], rr);
                rw = fmaf(g, CW[at - dj * cw_ - di], rw);
            }
            const float g = psf.gxy[dj + kxy];
            ur = fmaf(g, rr, ur);
            uw = fmaf(g, rw, uw);
        }
        // written after every thread has read phase-0 data? U is overwritten
        // only at lp, which no other thread reads in this phase.
        U[lp] = ur;
        Uw[lp] = uw;
    }
    __syncthreads();
    // phase 3: scatter
    if (interior)
        adjoint_scatter<KZ, PAIR, true>(vd, ti, kxy, kz, gz, U, Uw, addon, conf);
    else
        adjoint_scatter<KZ, PAIR, false>(vd, ti, kxy, kz, gz, U, Uw, addon, conf);
}

template <int KXY, int KZ, bool PAIR>
__global__ void __launch_bounds__(256, 3) k_adjoint(VolDims vd, const int32_t *__restrict__ desc,
                                                 const int32_t *__restrict__ fix, PsfTab psf,
                                                 Tiling tl, const float *__restrict__ r,
                                                 const float *__restrict__ w,
                                                 const uint8_t *__restrict__ pmask,
                                                 const float *__restrict__ pweight,
                                                 float *__restrict__ addon,
                                                 float *__restrict__ conf)
{
    extern __shared__ float sm[];
    adjoint_tile<KXY, KZ, PAIR>(tile_at(tl, blockIdx.x), vd, desc, fix, psf, tl, r, w, pmask, pweight, addon, conf, sm);
}

// The adjoint as a persistent work queue over listed (patch, tile) slots.
template <int KXY, int KZ, bool PAIR>
__global__ void __launch_bounds__(256, 3) k_adjoint_q(VolDims vd, const int32_t *__restrict__ desc,
                                                   const int32_t *__restrict__ fix, PsfTab psf,
                                                   Tiling tl, const float *__restrict__ r,
                                                   const float *__restrict__ w,
                                                   const uint8_t *__restrict__ pmask,
                                                   const float *__restrict__ pweight,
                                                   float *__restrict__ addon,
                                                   float *__restrict__ conf,
                                                   const int32_t *__restrict__ items, int n_items,
                                                   int *counter)
{
    extern __shared__ float sm[];
    __shared__ int cur;
    for (;;) {
        const int it = next_item(counter, &cur);
        if (it >= n_items) break;
        adjoint_tile<KXY, KZ, PAIR>(items[it], vd, desc, fix, psf, tl, r, w, pmask, pweight, addon, conf,
                                    sm);
        __syncthreads();
    }
}

__device__ __noinline__ bool ncc_of_sums(const double m[6], int min_valid, double &ncc, double &my, double &ms,
                                         double &sd, double &vs, double &n);

// EM tile partials {N, sum e^2, min e, max e} of a best_write tile from the
// threads' own counts, sums and extremes (the forward-model kernel's
// reductions).  sred: shared scratch of 128 floats.  Ends with a barrier.
__device__ __forceinline__ void best_part(int nval, float se2, float emin, float emax, const BestSim &bs,
                                          long long gid, float *sred)
{
    float acc[2] = {(float)nval, se2};
    const float mn = warp_min(emin), mx = warp_max(emax);
    float *rmn = sred + 64, *rmx = sred + 96;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        rmn[wid] = mn;
        rmx[wid] = mx;
    }
    block_sum_f<2>(acc, sred);
    if (threadIdx.x == 0) {
        float a = INFINITY, b = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a = fminf(a, rmn[w]);
            b = fmaxf(b, rmx[w]);
        }
        double *pt = bs.part + (size_t)gid * kPartStride;
        pt[0] = (double)acc[0];
        pt[1] = (double)acc[1];
        pt[2] = (double)a;
        pt[3] = (double)b;
    }
    __syncthreads();
}

// The kept residuals and flags are stored with the streaming (evict-first)
// policy: they are read again only after the registration, and must not push
// the persistent NCC kernel's gradient scratch out of L2.
// Forward model of a tile at the evaluated pose, written as the forward-model
// kernel writes it (BestSim): per pixel e = y - s and the valid flag, per tile
// {N, sum e^2, min e, max e} from the same per-thread order and reductions.
// sv(ci, cj) gives the simulated value of a valid pixel; B holds the PSF
// weights of the tile lattice.  sred: shared scratch of 128 floats.  Every
// thread of the block calls it; ends with a barrier.
template <class SV>
__device__ __forceinline__ void best_write(const TileInfo &ti, const Tiling &tl, int kxy, const float *gxy,
                                           const float *B, SV sv, const float *__restrict__ y, const BestSim &bs,
                                           long long gid, float *sred)
{
    float se2 = 0.f, emin = INFINITY, emax = -INFINITY;
    int nval = 0;
    const int np = ti.tw * ti.th;
    for (int pp = threadIdx.x; pp < np; pp += blockDim.x) {
        const int cj = qdiv(pp, ti.rtw), ci = pp - cj * ti.tw;
        const float den = inplane(B, ti.Lw, kxy, gxy, ci, cj);
        const size_t o = (size_t)ti.off + (size_t)(ti.j0 + cj) * ti.w + (ti.i0 + ci);
        const bool v = den > 0.f && member_ok(tl, o);
        const float s = v ? sv(ci, cj, den) : 0.f;
        const float e = v ? __ldg(y + o) - s : 0.f;
        __stcs(bs.e + o, e);
        __stcs(reinterpret_cast<signed char *>(bs.valid) + o, (signed char)(v ? 1 : 0));
        if (v) {
            se2 = fmaf(e, e, se2);
            emin = fminf(emin, e);
            emax = fmaxf(emax, e);
            ++nval;
        }
    }
    best_part(nval, se2, emin, emax, bs, gid, sred);
}

// best_write for a tile without samples: a table slot without a tile (the
// forward-model kernel zeroes its partials) or a pose outside the
// fixed-point range (every pixel invalid).
__device__ __forceinline__ void best_write_empty(bool has, const TileInfo &ti, const BestSim &bs, long long gid)
{
    double *pt = bs.part + (size_t)gid * kPartStride;
    if (!has) {
        if (threadIdx.x < kPartStride) pt[threadIdx.x] = 0.0;
        return;
    }
    const int np = ti.tw * ti.th;
    for (int pp = threadIdx.x; pp < np; pp += blockDim.x) {
        const int cj = qdiv(pp, ti.rtw), ci = pp - cj * ti.tw;
        const size_t o = (size_t)ti.off + (size_t)(ti.j0 + cj) * ti.w + (ti.i0 + ci);
        __stcs(bs.e + o, 0.f);
        __stcs(reinterpret_cast<signed char *>(bs.valid) + o, (signed char)0);
    }
    if (threadIdx.x == 0) {
        pt[0] = 0.0;
        pt[1] = 0.0;
        pt[2] = (double)INFINITY;
        pt[3] = (double)-INFINITY;
    }
}

// ----------------------------------------------------------------- K6a --
// Trilinear value and its gradient (voxel units) from one set of 8 loads.
template <bool FAST, class SRC>
__device__ __forceinline__ float tri_grad(const SRC &src, const VolDims &vd, unsigned qx, unsigned qy,
                                         unsigned qz, float gr[3])
{
    int bx, by, bz;
    float fx, fy, fz;
    split<FAST>(qx, vd.nx, bx, fx);
    split<FAST>(qy, vd.ny, by, fy);
    split<FAST>(qz, vd.nz, bz, fz);
    float v[8];
    cell_corners(src, vd, bx, by, bz, v);
    const float v000 = v[0], v100 = v[1], v010 = v[2], v110 = v[3];
    const float v001 = v[4], v101 = v[5], v011 = v[6], v111 = v[7];
    float dx00 = v100 - v000, dx10 = v110 - v010, dx01 = v101 - v001, dx11 = v111 - v011;
    float c00 = fmaf(fx, dx00, v000), c10 = fmaf(fx, dx10, v010);
    float c01 = fmaf(fx, dx01, v001), c11 = fmaf(fx, dx11, v011);
    float c0 = fmaf(fy, c10 - c00, c00), c1 = fmaf(fy, c11 - c01, c01);
    float gx0 = fmaf(fy, dx10 - dx00, dx00), gx1 = fmaf(fy, dx11 - dx01, dx01);
    gr[0] = fmaf(fz, gx1 - gx0, gx0);
    gr[1] = fmaf(fz, (c11 - c01) - (c10 - c00), c10 - c00);
    gr[2] = c1 - c0;
    return fmaf(fz, c1 - c0, c0);
}

// Through-plane sums of one lattice point with the trilinear gradient:
// a = sum g_z trilinear, b = sum g_z, ga = sum g_z grad, gb = sum g_z zeta grad
// over the in-volume samples.
template <int KZ, bool FAST, class SRC>
__device__ __forceinline__ void walk_grad(const SRC &src, const VolDims &vd, const TileInfo &ti,
                                          const unsigned q0[3], int kz_rt, const float *__restrict__ gz,
                                          float &a, float &b, float ga[3], float gb[3])
{
    const int kz = KZ >= 0 ? KZ : kz_rt;
#pragma unroll
    for (int z = -kz; z <= kz; ++z) {
        unsigned qx = q0[0] + (unsigned)z * ti.ez[0];
        unsigned qy = q0[1] + (unsigned)z * ti.ez[1];
        unsigned qz = q0[2] + (unsigned)z * ti.ez[2];
        if (!FAST && !inside(vd, qx, qy, qz)) continue;
        float gr[3];
        const float w = gz[z + kz];
        a = fmaf(w, tri_grad<FAST>(src, vd, qx, qy, qz, gr), a);
        b += w;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            ga[r] = fmaf(w, gr[r], ga[r]);
            gb[r] = fmaf(w * (float)z, gr[r], gb[r]);
        }
    }
}

// L2 policies of the gradient scratch.  The persistent kernels' slots (one
// per resident CTA, about 60 MB) are evict-last, so that the streamed patch
// pixels and kept residuals (evict-first) leave L2 before them and a slot is
// read back and discarded before it reaches DRAM; the chunked multi-tile
// path, whose scratch holds every tile of a chunk, stays evict-normal.
__device__ __forceinline__ uint64_t scratch_policy(bool keep)
{
    uint64_t pol;
    if (keep)
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    else
        asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Store / load of one gradient plane entry of the global scratch: kept in L2
// only (.cg), under the evict-last policy.
__device__ __forceinline__ void g_store(float *p, float v, uint64_t pol)
{
    asm volatile("st.global.cg.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ float g_load(const float *p, uint64_t pol)
{
    float v;
    asm volatile("ld.global.cg.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol) : "memory");
    return v;
}

// Gather pass of the NCC moments kernel: A, B into shared memory and the
// gradient sums GA, GB into G (FAST: interior tile).
template <int KZ, bool FAST, class SRC, bool KEEP_L2 = true>
__device__ __forceinline__ void moments_gather(const SRC src, const VolDims &vd,
                                               const TileInfo &ti, int kxy, int kz, int order,
                                               const float *__restrict__ gz, float *A, float *B,
                                               float *G, int Lmax)
{
    const uint64_t pol = scratch_policy(KEEP_L2);
    if (order != kAlongZeta) {
        for (int it = threadIdx.x; it < ti.L; it += blockDim.x) {
            int li, lj;
            lattice_coords(ti, order, it, li, lj);
            float a = 0.f, b = 0.f, ga[3] = {0.f, 0.f, 0.f}, gb[3] = {0.f, 0.f, 0.f};
            if (ti.ok) {
                unsigned q0[3];
                lattice_pos(ti, kxy, li, lj, q0);
                // border tile: warps whose walks are all inside take the FAST code
                if (FAST || __all_sync(__activemask(), walk_inside(vd, ti, q0, kz)))
                    walk_grad<KZ, true>(src, vd, ti, q0, kz, gz, a, b, ga, gb);
                else
                    walk_grad<KZ, false>(src, vd, ti, q0, kz, gz, a, b, ga, gb);
            }
            const int si = lj * ti.Lw + li;
            A[si] = a;
            B[si] = b;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                g_store(G + r * Lmax + si, ga[r], pol);
                g_store(G + (3 + r) * Lmax + si, gb[r], pol);
            }
        }
    } else {
        const int zl = threadIdx.x & 7, zeta = zl - kz;
        const bool zon = zl <= 2 * kz;
        const float w = zon ? gz[zl] : 0.f;
        const int ngrp = blockDim.x >> 3;
        for (int base = 0; base < ti.L; base += ngrp) {
            const int lp = base + (threadIdx.x >> 3);
            float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (zon && lp < ti.L) {
                unsigned q[3];
                const int lj = qdiv(lp, ti.rLw);
                lattice_pos(ti, kxy, lp - lj * ti.Lw, lj, q);
                unsigned qx = q[0] + (unsigned)zeta * ti.ez[0];
                unsigned qy = q[1] + (unsigned)zeta * ti.ez[1];
                unsigned qz = q[2] + (unsigned)zeta * ti.ez[2];
                if (FAST || inside(vd, qx, qy, qz)) {
                    float gr[3];
                    v[0] = w * tri_grad<FAST>(src, vd, qx, qy, qz, gr);
                    v[1] = w;
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        v[2 + r] = w * gr[r];
                        v[5 + r] = v[2 + r] * (float)zeta;
                    }
                }
            }
            // reduce-scatter over the group of 8 lanes: lane zl ends with the
            // group sum of v[zl] (halving the values kept at every step)
            const bool b2 = zl & 4, b1 = zl & 2, b0 = zl & 1;
            float w4[4], w2[2];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                w4[k] = (b2 ? v[k + 4] : v[k]) + __shfl_xor_sync(0xffffffffu, b2 ? v[k] : v[k + 4], 4);
#pragma unroll
            for (int k = 0; k < 2; ++k)
                w2[k] = (b1 ? w4[k + 2] : w4[k]) + __shfl_xor_sync(0xffffffffu, b1 ? w4[k] : w4[k + 2], 2);
            const float t = (b0 ? w2[1] : w2[0]) + __shfl_xor_sync(0xffffffffu, b0 ? w2[0] : w2[1], 1);
            if (lp < ti.L) {
                if (zl == 0) A[lp] = t;
                else if (zl == 1) B[lp] = t;
                else g_store(G + (zl - 2) * Lmax + lp, t, pol);
            }
        }
    }
}

// NCC moments of a tile: simulated pixel values (kept for K6b) and the sums
// {N, sum y, sum s, sum y^2, sum s^2, sum y s} (float64 per thread: the
// variances are differences of these sums and a constant patch must come
// out degenerate).  With gbuf, the same gather pass also computes the
// trilinear gradient of every sample and streams, per lattice point,
// GA = sum g_z grad and GB = sum g_z zeta grad (3 planes each, Lmax apart)
// to gbuf for K6b, which therefore gathers nothing.
template <int KXY, int KZ, class SRC, bool KEEP>
__global__ void __launch_bounds__(256, 4) k_ncc_moments(const SRC x, VolDims vd,
                                                     const int32_t *__restrict__ desc,
                                                     const int32_t *__restrict__ fix, PsfTab psf,
                                                     Tiling tl, long long tile_base,
                                                     const float *__restrict__ y,
                                                     const int32_t *__restrict__ active,
                                                     float *__restrict__ s_buf,
                                                     uint8_t *__restrict__ v_buf,
                                                     double *__restrict__ part,
                                                     float *__restrict__ gbuf, int Lmax, int min_valid,
                                                     BestSim bs)
{
    extern __shared__ float sm[];
    __shared__ double red[32 * 6];
    __shared__ int sh_best;
    const int kxy = KXY >= 0 ? KXY : psf.kxy;
    const int kz = KZ >= 0 ? KZ : psf.kz;
    const long long gid = tile_at(tl, tile_base + blockIdx.x);
    TileInfo ti;
    bool has = tile_setup_at(gid, desc, fix, tl, kxy, ti);
    double *pt = part + (size_t)gid * kPartStride;
    if (!has || (active && !active[ti.p])) {
        if (threadIdx.x < kPartStride) pt[threadIdx.x] = 0.0;
        if (KEEP && bs.mode == 1 && !has) best_write_empty(has, ti, bs, gid);
        return;
    }
    float *A = sm, *B = sm + ti.L;
    const float *gz = psf.gz[ti.stack];
    float *G = gbuf ? gbuf + (size_t)blockIdx.x * 6 * Lmax : nullptr;
    const int order = ti.ok ? pick_order(ti, kz) : kAlongCol;
    if (!G) {
        if (ti.ok) {
            if (tile_interior(ti, vd, kxy, kz))
                lattice_forward<KZ, true, SRC>(x, vd, ti, kxy, kz, gz, order, A, B);
            else
                lattice_forward<KZ, false, SRC>(x, vd, ti, kxy, kz, gz, order, A, B);
        } else {
            for (int lp = threadIdx.x; lp < ti.L; lp += blockDim.x) A[lp] = B[lp] = 0.f;
        }
    } else if (tile_interior(ti, vd, kxy, kz)) {
        moments_gather<KZ, true, SRC, false>(x, vd, ti, kxy, kz, order, gz, A, B, G, Lmax);
    } else {
        moments_gather<KZ, false, SRC, false>(x, vd, ti, kxy, kz, order, gz, A, B, G, Lmax);
    }
    __syncthreads();
    FFSum f1, f2, f3, f4, f5;
    int cnt = 0;
    const int np = ti.tw * ti.th;
    const bool keep_all = KEEP && bs.mode == 1;   // residuals written in this pass
    float se2 = 0.f, emin = INFINITY, emax = -INFINITY;
    for (int pp = threadIdx.x; pp < np; pp += blockDim.x) {
        const int cj = qdiv(pp, ti.rtw), ci = pp - cj * ti.tw;
        float num = inplane(A, ti.Lw, kxy, psf.gxy, ci, cj);
        float den = inplane(B, ti.Lw, kxy, psf.gxy, ci, cj);
        size_t o = (size_t)ti.off + (size_t)(ti.j0 + cj) * ti.w + (ti.i0 + ci);
        bool v = den > 0.f && member_ok(tl, o);
        float sv = v ? num / den : 0.f;
        if (s_buf) {   // kept for the separate gradient pass only
            s_buf[o] = sv;
            v_buf[o] = v ? 1 : 0;
        }
        float e = 0.f;
        if (v) {
            float a = __ldg(y + o);
            ++cnt;
            f1.add(a);
            f2.add(sv);
            f3.add_prod(a, a);
            f4.add_prod(sv, sv);
            f5.add_prod(a, sv);
            if (KEEP) {
                e = a - sv;
                se2 = fmaf(e, e, se2);
                emin = fminf(emin, e);
                emax = fmaxf(emax, e);
            }
        }
        if (keep_all) {
            __stcs(bs.e + o, e);
            __stcs(reinterpret_cast<signed char *>(bs.valid) + o, (signed char)(v ? 1 : 0));
        }
    }
    if (keep_all) best_part(cnt, se2, emin, emax, bs, gid, reinterpret_cast<float *>(red));
    FFSum fs[6] = {FFSum{(float)cnt, 0.f}, f1, f2, f3, f4, f5};   // counts <= 2^24: exact
    double m[6];
    block_sum_ff<6>(fs, m, red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) pt[k] = m[k];
        pt[6] = pt[7] = 0.0;
        if (KEEP && bs.mode) {   // one-tile patches only: the tile's sums are the patch's
            double ncc, my, ms, sd, vs, n;
            const bool ok = ncc_of_sums(m, min_valid, ncc, my, ms, sd, vs, n);
            sh_best = bs.mode == 2 && (bs.fixed || (ok ? ncc : 0.0) > bs.nbest[ti.p]);
        }
    }
    if (KEEP && bs.mode == 2) {
        __syncthreads();
        if (sh_best)
            best_write(ti, tl, kxy, psf.gxy, B,
                       [&](int ci, int cj, float den) { return inplane(A, ti.Lw, kxy, psf.gxy, ci, cj) / den; },
                       y, bs, gid, reinterpret_cast<float *>(red));
    }
}

// NCC of a patch from its tile moments (float64).  Returns false when
// degenerate (fewer than min_valid pixels or a constant patch).  Not inlined:
// the NCC kernels' acceptance test and k_ncc_finish must run the same
// instructions on the same sums.
__device__ __noinline__ bool ncc_of_sums(const double m[6], int min_valid, double &ncc, double &my, double &ms,
                            double &sd, double &vs, double &n)
{
    n = m[0];
    ncc = 0.0;
    if (n < (double)min_valid || n <= 0.0) return false;
    my = m[1] / n;
    ms = m[2] / n;
    double vy = m[3] / n - my * my;
    vs = m[4] / n - ms * ms;
    double cv = m[5] / n - my * ms;
    if (!(vy > 1e-12 * (my * my + 1.0)) || !(vs > 1e-12 * (ms * ms + 1.0))) return false;
    sd = sqrt(vy * vs);
    ncc = cv / sd;
    return true;
}

__device__ bool ncc_from_moments(const double *part, int p, int tpp, int min_valid, double &ncc,
                                 double &my, double &ms, double &sd, double &vs, double &n)
{
    double m[6] = {0, 0, 0, 0, 0, 0};
    for (int t = 0; t < tpp; ++t)
        for (int k = 0; k < 6; ++k) m[k] += part[((size_t)p * tpp + t) * kPartStride + k];
    return ncc_of_sums(m, min_valid, ncc, my, ms, sd, vs, n);
}

// Derivatives of the linear part of the patch transform, one 3x3 matrix per
// non-translation parameter: rigid (Rz Ry Rx, angles in degrees) the
// derivative of the product with respect to each angle, per degree;
// affine (I + D) the unit matrix of the entry D_rc.  float64 with
// math-library trigonometry: the gradient is not part of the
// integer-exact path.
__device__ void linear_derivs(const double *th, int n_params, double dL[9][9])
{
    if (n_params == 12) {
        for (int k = 0; k < 9; ++k)
            for (int e = 0; e < 9; ++e) dL[k][e] = e == k ? 1.0 : 0.0;
        return;
    }
    const double dg = 3.14159265358979323846 / 180.0;
    double sx, cx, sy, cy, sz, cz;
    sincos(th[3] * dg, &sx, &cx);
    sincos(th[4] * dg, &sy, &cy);
    sincos(th[5] * dg, &sz, &cz);
    const double Rx[9] = {1, 0, 0, 0, cx, -sx, 0, sx, cx};
    const double Ry[9] = {cy, 0, sy, 0, 1, 0, -sy, 0, cy};
    const double Rz[9] = {cz, -sz, 0, sz, cz, 0, 0, 0, 1};
    const double dRx[9] = {0, 0, 0, 0, -sx, -cx, 0, cx, -sx};
    const double dRy[9] = {-sy, 0, cy, 0, 0, 0, -cy, 0, -sy};
    const double dRz[9] = {-sz, -cz, 0, cz, -sz, 0, 0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        // angle a: x (rx), y (ry), z (rz); the derivative replaces that factor
        const double *Am = a == 2 ? dRz : Rz, *Bm = a == 1 ? dRy : Ry, *Cm = a == 0 ? dRx : Rx;
        double AB[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                AB[3 * r + c] = Am[3 * r] * Bm[c] + Am[3 * r + 1] * Bm[3 + c] + Am[3 * r + 2] * Bm[6 + c];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                dL[a][3 * r + c] =
                    (AB[3 * r] * Cm[c] + AB[3 * r + 1] * Cm[3 + c] + AB[3 * r + 2] * Cm[6 + c]) * dg;
    }
}

// Pose Jacobian of the sample positions (voxel units per parameter unit),
// column k: dq/dtheta_k = J1 (i - cu) + J2 (j - cv) + J4 zeta + J3 with
// (i, j) the patch pixel, (cu, cv) its centre; jc = {J1(3), J2(3), J4(3),
// J3(3)}.  Translations: J3 = columns of world_to_voxel.  Linear-part
// parameters: J = W dL S (the patch centre cancels), J4 scaled to one PSF
// step along the normal.
__device__ void pose_jacobian_col(const DevGeom *__restrict__ g, const int32_t *d, const double dL[9][9], int k,
                                  double jc[12])
{
    const double *S = g->p2w[d[0]];
    const double *W = g->w2v;
    if (k < 3) {
        for (int r = 0; r < 3; ++r) {
            jc[r] = jc[3 + r] = jc[6 + r] = 0.0;
            jc[9 + r] = W[4 * r + k];
        }
        return;
    }
    const double *D = dL[k - 3];
    const double n2 = S[2] * S[2] + S[6] * S[6] + S[10] * S[10];
    const double zs = g->dz / sqrt(n2);
    double WD[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) WD[3 * r + c] = W[4 * r] * D[c] + W[4 * r + 1] * D[3 + c] + W[4 * r + 2] * D[6 + c];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            const double q = WD[3 * r] * S[c] + WD[3 * r + 1] * S[4 + c] + WD[3 * r + 2] * S[8 + c];
            jc[3 * c + r] = c == 2 ? q * zs : q;
        }
        jc[9 + r] = 0.0;
    }
}

// Lattice phase of the NCC gradient: the transposed in-plane taps of the
// pixel coefficients (padded array Cp) give the lattice weight U; with the
// gradient sums GA, GB of the lattice point (planes of G, Lmax apart, read
// through L2) it accumulates M1 = sum U GA (i - cu), M2 = sum U GA (j - cv),
// M4 = sum U GB, M3 = sum U GA into mo[0..2], mo[3..5], mo[6..8], mo[9..11]
// (float32 per thread over its few lattice points).  The zero padding adds
// exact zeros where a tap falls outside the tile, so the sums equal those of
// a loop that skips them.
template <int KXY, bool KEEP_L2 = true>
__device__ __forceinline__ void grad_lattice_moments(const TileInfo &ti, int kxy_rt, const float *gxy,
                                                     const float *Cp, const float *G, int Lmax,
                                                     float mo[12])
{
    const int kxy = KXY >= 0 ? KXY : kxy_rt;
    const float cu = 0.5f * (float)(ti.w - 1), cv = 0.5f * (float)(ti.h - 1);
    const int cw = cpad_w(ti, kxy);
    const uint64_t pol = scratch_policy(KEEP_L2);
#pragma unroll
    for (int k = 0; k < 12; ++k) mo[k] = 0.f;
    for (int lp = threadIdx.x; lp < ti.L; lp += blockDim.x) {
        const int lj = qdiv(lp, ti.rLw), li = lp - lj * ti.Lw;
        const float *c0 = Cp + (lj + kxy) * cw + (li + kxy);
        float u = 0.f;
#pragma unroll
        for (int dj = -kxy; dj <= kxy; ++dj) {
            float rr = 0.f;
#pragma unroll
            for (int di = -kxy; di <= kxy; ++di) rr = fmaf(gxy[di + kxy], c0[-dj * cw - di], rr);
            u = fmaf(gxy[dj + kxy], rr, u);
        }
        if (u == 0.f) continue;
        const float di = (float)(ti.i0 - kxy + li) - cu, dj = (float)(ti.j0 - kxy + lj) - cv;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float s0 = u * g_load(G + r * Lmax + lp, pol);
            mo[r] = fmaf(s0, di, mo[r]);
            mo[3 + r] = fmaf(s0, dj, mo[3 + r]);
            mo[6 + r] = fmaf(u, g_load(G + (3 + r) * Lmax + lp, pol), mo[6 + r]);
            mo[9 + r] += s0;
        }
    }
}

// Plane stride of a persistent CTA's gradient slot: Lmax rounded up to 32
// floats, so that every slot starts on a 128-byte L2 line.
__host__ __device__ __forceinline__ int slot_stride(int Lmax)
{
    return (Lmax + 31) & ~31;
}

// Drop a CTA's gradient slot (6 planes of stride Gs, 128-byte aligned) from L2
// without writing it back: its values are dead once the tile's gradient
// moments are summed, and a write-back would only cost HBM bandwidth.
// discard.global.L2 acts as a write of undefined values, so the callers put a
// barrier after the last read and another before the slot is written again.
__device__ __forceinline__ void discard_slot(float *G, int Gs)
{
    for (int l = threadIdx.x * 32; l < 6 * Gs; l += blockDim.x * 32)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(G + l) : "memory");
}

// ----------------------------------------------------------------- K6b --
// Pose gradient of NCC from the gradient sums K6a streamed to gbuf.
// dNCC/ds_i = ((y_i - my)/sd - ncc (s_i - ms)/vs)/N; pixel coefficient
// c_i = dNCC/ds_i / den_i; the transposed in-plane taps give lattice weights
// U; the moments M1 = sum U GA (i - cu), M2 = sum U GA (j - cv),
// M3 = sum U GA, M4 = sum U GB (float32 per thread over its few lattice
// points, float64 across threads), written per tile; k_ncc_finish contracts
// them with the pose Jacobian once per patch.
template <int KXY, int KZ>
__global__ void __launch_bounds__(256) k_ncc_grad(VolDims vd, const DevGeom *__restrict__ g,
                                                  const int32_t *__restrict__ desc,
                                                  const int32_t *__restrict__ fix, PsfTab psf,
                                                  Tiling tl, long long tile_base,
                                                  const float *__restrict__ y,
                                                  const double *__restrict__ poses,
                                                  const int32_t *__restrict__ active,
                                                  const float *__restrict__ s_buf,
                                                  const uint8_t *__restrict__ v_buf,
                                                  const double *__restrict__ part,
                                                  double *__restrict__ gpart,
                                                  const float *__restrict__ gbuf, int Lmax,
                                                  int min_valid)
{
    extern __shared__ float sm[];
    __shared__ double red[32 * 12];
    __shared__ float sh_coef[4];
    __shared__ int sh_ok;
    const int kxy = KXY >= 0 ? KXY : psf.kxy;
    const int kz = KZ >= 0 ? KZ : psf.kz;
    const long long gid = tile_at(tl, tile_base + blockIdx.x);
    TileInfo ti;
    bool has = tile_setup_at(gid, desc, fix, tl, kxy, ti);
    double *gp = gpart + (size_t)gid * kGradStride;
    if (!has || !ti.ok || (active && !active[ti.p])) {
        if (threadIdx.x < kGradStride) gp[threadIdx.x] = 0.0;
        return;
    }
    if (threadIdx.x == 0) {
        double ncc, my, ms, sd, vs, n;
        bool ok = ncc_from_moments(part, ti.p, tl.tpp, min_valid, ncc, my, ms, sd, vs, n);
        sh_ok = ok;
        if (ok) {
            sh_coef[0] = (float)(1.0 / (n * sd));
            sh_coef[1] = (float)(ncc / (n * vs));
            sh_coef[2] = (float)my;
            sh_coef[3] = (float)ms;
        }
    }
    __syncthreads();
    if (!sh_ok) {
        if (threadIdx.x < kGradStride) gp[threadIdx.x] = 0.0;
        return;
    }
    const int np = ti.tw * ti.th;
    float *U = sm, *C = sm + ti.L;
    lattice_forward<KZ>(PlainVol{nullptr}, vd, ti, kxy, kz, psf.gz[ti.stack], kAlongCol, nullptr, U);
    __syncthreads();
    const float a_sc = sh_coef[0], b_sc = sh_coef[1], my = sh_coef[2], ms = sh_coef[3];
    cpad_border(ti, kxy, C);
    for (int pp = threadIdx.x; pp < np; pp += blockDim.x) {
        const int cj = qdiv(pp, ti.rtw), ci = pp - cj * ti.tw;
        size_t o = (size_t)ti.off + (size_t)(ti.j0 + cj) * ti.w + (ti.i0 + ci);
        float c = 0.f;
        if (v_buf[o]) {
            float den = inplane(U, ti.Lw, kxy, psf.gxy, ci, cj);
            c = (a_sc * (__ldg(y + o) - my) - b_sc * (s_buf[o] - ms)) / den;
        }
        C[cpad_at(ti, kxy, ci, cj)] = c;
    }
    __syncthreads();
    float mo[12];
    grad_lattice_moments<KXY, false>(ti, kxy, psf.gxy, C, gbuf + (size_t)blockIdx.x * 6 * Lmax, Lmax, mo);
    double mom[12];
    block_sum_fd<12>(mo, mom, red);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 12; ++k) gp[k] = mom[k];
        for (int k = 12; k < kGradStride; ++k) gp[k] = 0.0;
    }
}

// K6a + K6b in one persistent kernel for one-tile patches (every patch side
// <= the tile side): the CTA holds the whole patch, so once its moments are
// reduced it knows the patch's NCC coefficients and finishes the gradient
// moments itself.  The gradient sums GA, GB of the current tile go to the
// CTA's own slot of the scratch (6 Lmax floats, rewritten for every tile and
// read back by the same CTA through L2), so they never make an HBM round
// trip, and no simulated pixel values are stored.  Grid: at most the number
// of co-resident CTAs; CTA b takes tiles b, b + grid, ...
template <int KXY, int KZ, class SRC>
__global__ void __launch_bounds__(256, 4) k_ncc_fused(const SRC x, VolDims vd,
                                                      const int32_t *__restrict__ desc,
                                                      const int32_t *__restrict__ fix, PsfTab psf,
                                                      Tiling tl, long long n_tiles,
                                                      const float *__restrict__ y,
                                                      const int32_t *__restrict__ active,
                                                      double *__restrict__ part,
                                                      double *__restrict__ gpart,
                                                      float *__restrict__ scratch, int Lmax,
                                                      int min_valid, BestSim bs, int *__restrict__ counter)
{
    extern __shared__ float sm[];
    __shared__ double red[32 * 12];
    __shared__ float sh_coef[4];
    __shared__ int sh_ok, sh_best;
    const int kxy = KXY >= 0 ? KXY : psf.kxy;
    const int kz = KZ >= 0 ? KZ : psf.kz;
    const int Gs = slot_stride(Lmax);
    float *G = scratch + (size_t)blockIdx.x * 6 * Gs;
    float *A = sm, *B = sm + Lmax, *C = sm + 2 * Lmax;
    __shared__ int cur;
    for (;;) {
        // tiles from a shared counter (CTAs that finish early take more);
        // the barrier first: every thread has read the previous index
        __syncthreads();
        if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
        __syncthreads();
        if (cur >= n_tiles) break;
        const long long gid = tile_at(tl, cur);
        TileInfo ti;
        const bool has = tile_setup_at(gid, desc, fix, tl, kxy, ti);
        double *pt = part + (size_t)gid * kPartStride;
        double *gp = gpart + (size_t)gid * kGradStride;
        // outside the fixed-point range every pixel is invalid: zero moments
        if (!has || !ti.ok || (active && !active[ti.p])) {
            if (threadIdx.x < kPartStride) pt[threadIdx.x] = 0.0;
            if (threadIdx.x < kGradStride) gp[threadIdx.x] = 0.0;
            // no samples: every pixel invalid, NCC 0 (accepted by the same rule)
            if (bs.mode == 1 && (!has || !ti.ok)) best_write_empty(has, ti, bs, gid);
            if (bs.mode == 2 && has && !ti.ok && !(active && !active[ti.p]) && (bs.fixed || 0.0 > bs.nbest[ti.p]))
                best_write_empty(true, ti, bs, gid);
            continue;
        }
        const float *gz = psf.gz[ti.stack];
        const int order = pick_order(ti, kz);
        if (tile_interior(ti, vd, kxy, kz))
            moments_gather<KZ, true, SRC>(x, vd, ti, kxy, kz, order, gz, A, B, G, Gs);
        else
            moments_gather<KZ, false, SRC>(x, vd, ti, kxy, kz, order, gz, A, B, G, Gs);
        __syncthreads();
        FFSum f1, f2, f3, f4, f5;
        int cnt = 0;
        const int np = ti.tw * ti.th;
        // first evaluation keeping the forward model: residuals written in this pass
        const bool keep_all = bs.mode == 1;
        float se2 = 0.f, emin = INFINITY, emax = -INFINITY;
        cpad_border(ti, kxy, C);
        for (int pp = threadIdx.x; pp < np; pp += blockDim.x) {
            const int cj = qdiv(pp, ti.rtw), ci = pp - cj * ti.tw;
            const float den = inplane(B, ti.Lw, kxy, psf.gxy, ci, cj);
            const size_t o = (size_t)ti.off + (size_t)(ti.j0 + cj) * ti.w + (ti.i0 + ci);
            const bool v = den > 0.f && member_ok(tl, o);
            float e = 0.f;
            if (v) {
                const float sv = inplane(A, ti.Lw, kxy, psf.gxy, ci, cj) / den;
                C[cpad_at(ti, kxy, ci, cj)] = sv;   // kept for the gradient pass
                const float a = __ldg(y + o);
                ++cnt;
                f1.add(a);
                f2.add(sv);
                f3.add_prod(a, a);
                f4.add_prod(sv, sv);
                f5.add_prod(a, sv);
                e = a - sv;
                se2 = fmaf(e, e, se2);
                emin = fminf(emin, e);
                emax = fmaxf(emax, e);
            }
            if (keep_all) {
                __stcs(bs.e + o, e);
                __stcs(reinterpret_cast<signed char *>(bs.valid) + o, (signed char)(v ? 1 : 0));
            }
        }
        if (keep_all) best_part(cnt, se2, emin, emax, bs, gid, reinterpret_cast<float *>(red));
        FFSum fs[6] = {FFSum{(float)cnt, 0.f}, f1, f2, f3, f4, f5};   // counts <= 2^24: exact
        double m[6];
        block_sum_ff<6>(fs, m, red);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) pt[k] = m[k];
            pt[6] = pt[7] = 0.0;
            double ncc, my, ms, sd, vs, n;
            const bool ok = ncc_of_sums(m, min_valid, ncc, my, ms, sd, vs, n);
            sh_ok = ok;
            if (ok) {
                sh_coef[0] = (float)(1.0 / (n * sd));
                sh_coef[1] = (float)(ncc / (n * vs));
                sh_coef[2] = (float)my;
                sh_coef[3] = (float)ms;
            }
            // the registration's acceptance test on the NCC k_ncc_finish reports
            const bool decide = bs.mode == 2 || bs.grad_if_accepted;   // bs.nbest is set then
            const bool accepted = decide && (bs.fixed || (ok ? ncc : 0.0) > bs.nbest[ti.p]);
            sh_best = bs.mode == 2 && accepted;
            // a rejected trial's gradient is never used
            if (bs.grad_if_accepted && !accepted) sh_ok = 0;
        }
        __syncthreads();
        if (sh_best)
            best_write(ti, tl, kxy, psf.gxy, B, [&](int ci, int cj, float) { return C[cpad_at(ti, kxy, ci, cj)]; },
                       y, bs, gid, reinterpret_cast<float *>(red));
        if (!sh_ok) {
            if (threadIdx.x < kGradStride) gp[threadIdx.x] = 0.0;
            discard_slot(G, Gs);
            __syncthreads();
            continue;
        }
        // dNCC/ds per pixel over its PSF weight (as K6b), from the same A, B
        const float a_sc = sh_coef[0], b_sc = sh_coef[1], my = sh_coef[2], ms = sh_coef[3];
        for (int pp = threadIdx.x; pp < np; pp += blockDim.x) {
            const int cj = qdiv(pp, ti.rtw), ci = pp - cj * ti.tw;
            const float den = inplane(B, ti.Lw, kxy, psf.gxy, ci, cj);
            const size_t o = (size_t)ti.off + (size_t)(ti.j0 + cj) * ti.w + (ti.i0 + ci);
            const int at = cpad_at(ti, kxy, ci, cj);
            float c = 0.f;
            if (den > 0.f && member_ok(tl, o)) c = (a_sc * (__ldg(y + o) - my) - b_sc * (C[at] - ms)) / den;
            C[at] = c;
        }
        __syncthreads();
        float mo[12];
        grad_lattice_moments<KXY>(ti, kxy, psf.gxy, C, G, Gs, mo);
        double mom[12];
        block_sum_fd<12>(mo, mom, red);   // ends with a barrier: A, B, C, G free for the next tile
        if (threadIdx.x == 0) {
            for (int k = 0; k < 12; ++k) gp[k] = mom[k];
            for (int k = 12; k < kGradStride; ++k) gp[k] = 0.0;
        }
        discard_slot(G, Gs);
        __syncthreads();
    }
}

// Pose vector-Jacobian product of the forward model (backward pass of a
// differentiable simulate): per tile, the gradient moments of
// sum_pix r_pix s_pix, i.e. the lattice phase of the NCC gradient with the
// pixel coefficient r / den.  Tile moments add over a patch's tiles, so any
// tiling works.  Persistent like k_ncc_fused: one scratch slot per CTA.
template <int KXY, int KZ, class SRC>
__global__ void __launch_bounds__(256, 4) k_pose_vjp(const SRC x, VolDims vd,
                                                     const int32_t *__restrict__ desc,
                                                     const int32_t *__restrict__ fix, PsfTab psf,
                                                     Tiling tl, long long n_tiles,
                                                     const float *__restrict__ r,
                                                     double *__restrict__ gpart,
                                                     float *__restrict__ scratch, int Lmax,
                                                     int *__restrict__ counter)
{
    extern __shared__ float sm[];
    __shared__ double red[32 * 12];
    const int kxy = KXY >= 0 ? KXY : psf.kxy;
    const int kz = KZ >= 0 ? KZ : psf.kz;
    const int Gs = slot_stride(Lmax);
    float *G = scratch + (size_t)blockIdx.x * 6 * Gs;
    float *A = sm, *B = sm + Lmax, *C = sm + 2 * Lmax;
    __shared__ int cur;
    for (;;) {
        // tiles from a shared counter, as in k_ncc_fused
        __syncthreads();
        if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
        __syncthreads();
        if (cur >= n_tiles) break;
        const long long gid = tile_at(tl, cur);
        TileInfo ti;
        const bool has = tile_setup_at(gid, desc, fix, tl, kxy, ti);
        double *gp = gpart + (size_t)gid * kGradStride;
        if (!has || !ti.ok) {
            if (threadIdx.x < kGradStride) gp[threadIdx.x] = 0.0;
            continue;
        }
        const float *gz = psf.gz[ti.stack];
        const int order = pick_order(ti, kz);
        if (tile_interior(ti, vd, kxy, kz))
            moments_gather<KZ, true, SRC>(x, vd, ti, kxy, kz, order, gz, A, B, G, Gs);
        else
            moments_gather<KZ, false, SRC>(x, vd, ti, kxy, kz, order, gz, A, B, G, Gs);
        __syncthreads();
        const int np = ti.tw * ti.th;
        cpad_border(ti, kxy, C);
        for (int pp = threadIdx.x; pp < np; pp += blockDim.x) {
            const int cj = qdiv(pp, ti.rtw), ci = pp - cj * ti.tw;
            const float den = inplane(B, ti.Lw, kxy, psf.gxy, ci, cj);
            const size_t o = (size_t)ti.off + (size_t)(ti.j0 + cj) * ti.w + (ti.i0 + ci);
            float c = 0.f;
            if (den > 0.f && member_ok(tl, o)) c = __ldg(r + o) / den;
            C[cpad_at(ti, kxy, ci, cj)] = c;
        }
        __syncthreads();
        float mo[12];
        grad_lattice_moments<KXY>(ti, kxy, psf.gxy, C, G, Gs, mo);
        double mom[12];
        block_sum_fd<12>(mo, mom, red);   // ends with a barrier: A, B, C, G free for the next tile
        if (threadIdx.x == 0) {
            for (int k = 0; k < 12; ++k) gp[k] = mom[k];
            for (int k = 12; k < kGradStride; ++k) gp[k] = 0.0;
        }
        discard_slot(G, Gs);
        __syncthreads();
    }
}

// Per patch: NCC from the tile moments, and the pose gradient as the
// contraction of the summed gradient moments with the pose Jacobian.
__global__ void k_ncc_finish(const DevGeom *__restrict__ g, int n_params, int n, int tpp,
                             const int32_t *__restrict__ desc, const double *__restrict__ poses,
                             const double *__restrict__ part, const double *__restrict__ gpart,
                             int min_valid, double *__restrict__ ncc, double *__restrict__ grad)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    bool ok = true;   // part == null: gradient moments only (pose VJP)
    if (part) {
        double v, my, ms, sd, vs, nn;
        ok = ncc_from_moments(part, p, tpp, min_valid, v, my, ms, sd, vs, nn);
        ncc[p] = ok ? v : 0.0;
    }
    if (!grad) return;
    double *gr = grad + (size_t)n_params * p;
    if (!ok) {
        for (int k = 0; k < n_params; ++k) gr[k] = 0.0;
        return;
    }
    double mom[12];
    for (int k = 0; k < 12; ++k) {
        double s = 0.0;
        for (int t = 0; t < tpp; ++t) s += gpart[((size_t)p * tpp + t) * kGradStride + k];
        mom[k] = s;
    }
    const int32_t *d = desc + 8 * (size_t)p;
    if (n_params == 12) {
        // affine: the derivative of the linear part by entry (a, b) is the
        // unit matrix E_ab, so column k = 3 + 3a + b of the Jacobian is
        // W[:, a] S[b, :] (the values pose_jacobian_col forms from E_ab,
        // whose other products are exact zeros)
        const double *S = g->p2w[d[0]];
        const double *W = g->w2v;
        const double zs = g->dz / sqrt(S[2] * S[2] + S[6] * S[6] + S[10] * S[10]);
        for (int k = 0; k < 12; ++k) {
            double jc[12];
            if (k < 3) {
                for (int r = 0; r < 3; ++r) {
                    jc[r] = jc[3 + r] = jc[6 + r] = 0.0;
                    jc[9 + r] = W[4 * r + k];
                }
            } else {
                const int ea = (k - 3) / 3, eb = (k - 3) % 3;
                for (int r = 0; r < 3; ++r) {
                    for (int c = 0; c < 3; ++c) {
                        const double q = W[4 * r + ea] * S[4 * eb + c];
                        jc[3 * c + r] = c == 2 ? q * zs : q;
                    }
                    jc[9 + r] = 0.0;
                }
            }
            double gsum = 0.0;
            for (int r = 0; r < 3; ++r)
                gsum += jc[r] * mom[r] + jc[3 + r] * mom[3 + r] + jc[6 + r] * mom[6 + r] + jc[9 + r] * mom[9 + r];
            gr[k] = gsum;
        }
        return;
    }
    double dL[9][9];
    linear_derivs(poses + (size_t)n_params * p, n_params, dL);
    for (int k = 0; k < n_params; ++k) {
        double jc[12];
        pose_jacobian_col(g, d, dL, k, jc);
        double gsum = 0.0;
        for (int r = 0; r < 3; ++r)
            gsum += jc[r] * mom[r] + jc[3 + r] * mom[3 + r] + jc[6 + r] * mom[6 + r] + jc[9 + r] * mom[9 + r];
        gr[k] = gsum;
    }
}

size_t smem_forward(const Tiling &tl, int kxy)
{
    size_t L = (size_t)(tl.T + 2 * kxy) * (tl.T + 2 * kxy);
    return 2 * L * sizeof(float);
}

size_t smem_adjoint(const Tiling &tl, int kxy)
{
    size_t L = (size_t)(tl.T + 2 * kxy) * (tl.T + 2 * kxy);
    size_t Cp = (size_t)(tl.T + 4 * kxy) * (tl.T + 4 * kxy);   // padded pixel coefficients
    return (2 * L + 2 * Cp) * sizeof(float);
}

// Quad copy of the volume for QuadVol gathers: q[i] = (x[i], x[i + 1],
// x[i + nx], x[i + nx + 1]) for every voxel i with bx < nx - 1 and
// by < ny - 1 (the cells a sample can address); the last column and row
// are never read and hold their own voxel four times.
__global__ void k_build_quad(const float *__restrict__ x, float4 *__restrict__ q, int nx, int ny,
                             unsigned n)
{
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned bx = i % (unsigned)nx, by = (i / (unsigned)nx) % (unsigned)ny;
        const unsigned dx = bx + 1 < (unsigned)nx ? 1u : 0u;
        const unsigned dy = by + 1 < (unsigned)ny ? (unsigned)nx : 0u;
        q[i] = make_float4(__ldg(x + i), __ldg(x + i + dx), __ldg(x + i + dy), __ldg(x + i + dy + dx));
    }
}

template <typename K>
cudaError_t prep(K kern, size_t smem)
{
    if (smem > 48 * 1024) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

}  // namespace

// Launchers: the (kxy, kz) = (1, 3) specialisation serves the default PSF;
// every other setting takes the runtime-loop instantiation.

// Grid of a persistent kernel: every co-resident CTA, at most n_items.
template <typename K>
cudaError_t persistent_grid(K kern, size_t smem, int n_items, unsigned *grid)
{
    int dev = 0, nsm = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem)) != cudaSuccess) return e;
    long long g = (long long)(per_sm > 0 ? per_sm : 1) * nsm;
    *grid = (unsigned)(g < n_items ? g : n_items);
    return cudaSuccess;
}

cudaError_t launch_simulate(const DevGeom *, const PsfTab &psf, const Tiling &tl, int nx, int ny,
                            int nz, const float *x, const float4 *quad, const int32_t *desc,
                            const int32_t *fix, int n, const float *y, float *out, uint8_t *valid,
                            double *part, cudaStream_t st, const WorkQueue *wq)
{
    if (n <= 0) return cudaSuccess;
    VolDims vd = vol_dims(nx, ny, nz);
    size_t smem = smem_forward(tl, psf.kxy);
    dim3 grid((unsigned)n * tl.tpp), block(256);
    cudaError_t e;
    if (wq && wq->items) {
        if (wq->n_items <= 0) return cudaSuccess;
        if ((e = cudaMemsetAsync(wq->counter, 0, sizeof(int), st)) != cudaSuccess) return e;
    }
#define PVR_SIM(KX, KZv, SRCT, src)                                                                  \
    do {                                                                                          \
        if (wq && wq->items) {                                                                    \
            unsigned pg;                                                                          \
            if ((e = prep(k_simulate_q<KX, KZv, SRCT>, smem)) != cudaSuccess) return e;            \
            if ((e = persistent_grid(k_simulate_q<KX, KZv, SRCT>, smem, wq->n_items, &pg)) != cudaSuccess) \
                return e;                                                                         \
            k_simulate_q<KX, KZv, SRCT><<<pg, block, smem, st>>>(src, vd, desc, fix, psf, tl, y, out, \
                                                                 valid, part, wq->items, wq->n_items, \
                                                                 wq->counter);                    \
        } else {                                                                                  \
            if ((e = prep(k_simulate<KX, KZv, SRCT>, smem)) != cudaSuccess) return e;              \
            k_simulate<KX, KZv, SRCT><<<grid, block, smem, st>>>(src, vd, desc, fix, psf, tl, y, out, \
                                                                 valid, part);                    \
        }                                                                                         \
    } while (0)
    const bool fast = psf.kxy == 1 && psf.kz == 3;
    if (quad) {
        if (fast) PVR_SIM(1, 3, QuadVol, QuadVol{quad});
        else PVR_SIM(-1, -1, QuadVol, QuadVol{quad});
    } else {
        if (fast) PVR_SIM(1, 3, PlainVol, PlainVol{x});
        else PVR_SIM(-1, -1, PlainVol, PlainVol{x});
    }
#undef PVR_SIM
    return cudaGetLastError();
}

cudaError_t launch_build_quad(const float *x, float4 *quad, int nx, int ny, int nz, cudaStream_t st)
{
    const unsigned n = (unsigned)nx * (unsigned)ny * (unsigned)nz;
    int dev = 0, nsm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    unsigned blocks = (n + 255) / 256, cap = 8u * (unsigned)nsm;
    k_build_quad<<<blocks < cap ? blocks : cap, 256, 0, st>>>(x, quad, nx, ny, n);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const PsfTab &psf, const Tiling &tl, int nx, int ny, int nz,
                           const int32_t *desc, const int32_t *fix, int n, const float *r,
                           const float *w, const uint8_t *pmask, float *addon, float *conf,
                           int pair, cudaStream_t st, const WorkQueue *wq, const float *pweight)
{
    if (n <= 0) return cudaSuccess;
    VolDims vd = vol_dims(nx, ny, nz);
    size_t smem = smem_adjoint(tl, psf.kxy);
    dim3 grid((unsigned)n * tl.tpp), block(256);
    cudaError_t e;
    if (wq && wq->items) {
        if (wq->n_items <= 0) return cudaSuccess;
        if ((e = cudaMemsetAsync(wq->counter, 0, sizeof(int), st)) != cudaSuccess) return e;
    }
#define PVR_ADJ(KX, KZv, PR)                                                                          \
    do {                                                                                              \
        if (wq && wq->items) {                                                                        \
            unsigned pg;                                                                              \
            if ((e = prep(k_adjoint_q<KX, KZv, PR>, smem)) != cudaSuccess) return e;                  \
            if ((e = persistent_grid(k_adjoint_q<KX, KZv, PR>, smem, wq->n_items, &pg)) != cudaSuccess) \
                return e;                                                                             \
            k_adjoint_q<KX, KZv, PR><<<pg, block, smem, st>>>(vd, desc, fix, psf, tl, r, w, pmask,    \
                                                              pweight, addon, conf, wq->items,        \
                                                              wq->n_items,                            \
                                                              wq->counter);                           \
        } else {                                                                                      \
            if ((e = prep(k_adjoint<KX, KZv, PR>, smem)) != cudaSuccess) return e;                    \
            k_adjoint<KX, KZv, PR><<<grid, block, smem, st>>>(vd, desc, fix, psf, tl, r, w, pmask,    \
                                                              pweight, addon, conf);                  \
        }                                                                                             \
    } while (0)
    const bool fast = psf.kxy == 1 && psf.kz == 3;
    if (fast && pair) PVR_ADJ(1, 3, true);
    else if (fast) PVR_ADJ(1, 3, false);
    else if (pair) PVR_ADJ(-1, -1, true);
    else PVR_ADJ(-1, -1, false);
#undef PVR_ADJ
    return cudaGetLastError();
}

cudaError_t launch_ncc_grad(const DevGeom *g, const PsfTab &psf, const Tiling &tl, int nx, int ny,
                            int nz, const float *xplain, const float4 *quad, const float *y,
                            const int32_t *desc, const int32_t *fix, const double *poses, int n,
                            float *s_buf,
                            uint8_t *v_buf, double *part, double *gpart, const int32_t *active,
                            int min_valid, float *gbuf, long long gbuf_tiles, int *counter, cudaStream_t st,
                            const BestSim &bs_in)
{
    // the best-pose forward model is kept for one-tile patches only (the
    // acceptance test needs the whole patch's NCC inside the tile's block)
    BestSim bs = bs_in;
    if (tl.tpp != 1) bs.mode = 0;
    if (n <= 0) return cudaSuccess;
    VolDims vd = vol_dims(nx, ny, nz);
    const QuadVol x{quad};
    size_t smem = smem_forward(tl, psf.kxy);
    const int Lmax = (tl.T + 2 * psf.kxy) * (tl.T + 2 * psf.kxy);
    const int Cmax = (tl.T + 4 * psf.kxy) * (tl.T + 4 * psf.kxy);   // padded coefficient array
    size_t smem2 = (size_t)(Lmax + Cmax) * sizeof(float);
    const long long total = (long long)n * tl.tpp;
    const bool fast = psf.kxy == 1 && psf.kz == 3;
    cudaError_t e;
    if (gpart && tl.tpp == 1) {
        // one-tile patches: the fused persistent kernel, one scratch slot per
        // CTA.  It gathers from the plain volume: the scratch slots in flight
        // (about 60 MB) then share L2 with 50 MB of volume instead of the
        // 200 MB quad copy, and stay on chip.
        const PlainVol xp{xplain};
        size_t smem3 = (size_t)(2 * Lmax + Cmax) * sizeof(float);
        int dev = 0, nsm = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if (fast) {
            if ((e = prep(k_ncc_fused<1, 3, PlainVol>, smem3)) != cudaSuccess) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ncc_fused<1, 3, PlainVol>, 256, smem3);
        } else {
            if ((e = prep(k_ncc_fused<-1, -1, PlainVol>, smem3)) != cudaSuccess) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ncc_fused<-1, -1, PlainVol>, 256, smem3);
        }
        if (e != cudaSuccess) return e;
        long long grid = (long long)(per_sm > 0 ? per_sm : 1) * nsm;
        if (grid > total) grid = total;
        const long long slots = gbuf_tiles * Lmax / slot_stride(Lmax);   // padded slots in the scratch
        if (grid > slots) grid = slots;
        if (grid <= 0) return cudaErrorInvalidValue;
        if ((e = cudaMemsetAsync(counter, 0, sizeof(int), st)) != cudaSuccess) return e;
        if (fast)
            k_ncc_fused<1, 3, PlainVol><<<(unsigned)grid, 256, smem3, st>>>(xp, vd, desc, fix, psf, tl, total, y, active,
                                                                  part, gpart, gbuf, Lmax, min_valid, bs, counter);
        else
            k_ncc_fused<-1, -1, PlainVol><<<(unsigned)grid, 256, smem3, st>>>(xp, vd, desc, fix, psf, tl, total, y,
                                                                    active, part, gpart, gbuf, Lmax,
                                                                    min_valid, bs, counter);
        return cudaGetLastError();
    }
    // chunks of whole patches that fit the gradient scratch
    long long chunk = gpart ? (gbuf_tiles / tl.tpp) * tl.tpp : total;
    if (chunk <= 0) return cudaErrorInvalidValue;
    const bool keep = bs.mode != 0;
    if (fast) {
        if ((e = prep(k_ncc_moments<1, 3, QuadVol, false>, smem)) != cudaSuccess) return e;
        if ((e = prep(k_ncc_moments<1, 3, QuadVol, true>, smem)) != cudaSuccess) return e;
        if ((e = prep(k_ncc_grad<1, 3>, smem2)) != cudaSuccess) return e;
    } else {
        if ((e = prep(k_ncc_moments<-1, -1, QuadVol, false>, smem)) != cudaSuccess) return e;
        if ((e = prep(k_ncc_moments<-1, -1, QuadVol, true>, smem)) != cudaSuccess) return e;
        if ((e = prep(k_ncc_grad<-1, -1>, smem2)) != cudaSuccess) return e;
    }
    if (!gpart) s_buf = nullptr, v_buf = nullptr;
    for (long long base = 0; base < total; base += chunk) {
        unsigned grid = (unsigned)((total - base) < chunk ? (total - base) : chunk);
        float *gb = gpart ? gbuf : nullptr;
        if (fast && keep)
            k_ncc_moments<1, 3, QuadVol, true><<<grid, 256, smem, st>>>(x, vd, desc, fix, psf, tl, base, y, active,
                                                                     s_buf, v_buf, part, gb, Lmax, min_valid, bs);
        else if (fast)
            k_ncc_moments<1, 3, QuadVol, false><<<grid, 256, smem, st>>>(x, vd, desc, fix, psf, tl, base, y, active,
                                                                      s_buf, v_buf, part, gb, Lmax, min_valid, bs);
        else if (keep)
            k_ncc_moments<-1, -1, QuadVol, true><<<grid, 256, smem, st>>>(x, vd, desc, fix, psf, tl, base, y,
                                                                       active, s_buf, v_buf, part, gb, Lmax,
                                                                       min_valid, bs);
        else
            k_ncc_moments<-1, -1, QuadVol, false><<<grid, 256, smem, st>>>(x, vd, desc, fix, psf, tl, base, y,
                                                                        active, s_buf, v_buf, part, gb, Lmax,
                                                                        min_valid, bs);
        if (!gpart) continue;
        if (fast)
            k_ncc_grad<1, 3><<<grid, 256, smem2, st>>>(vd, g, desc, fix, psf, tl, base, y, poses, active,
                                                       s_buf, v_buf, part, gpart, gbuf, Lmax, min_valid);
        else
            k_ncc_grad<-1, -1><<<grid, 256, smem2, st>>>(vd, g, desc, fix, psf, tl, base, y, poses, active,
                                                         s_buf, v_buf, part, gpart, gbuf, Lmax, min_valid);
    }
    return cudaGetLastError();
}

cudaError_t launch_pose_vjp(const PsfTab &psf, const Tiling &tl, int nx, int ny, int nz,
                            const float *xplain, const float *r, const int32_t *desc,
                            const int32_t *fix, int n, double *gpart, float *gbuf,
                            long long gbuf_tiles, int *counter, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    VolDims vd = vol_dims(nx, ny, nz);
    const PlainVol x{xplain};
    const int Lmax = (tl.T + 2 * psf.kxy) * (tl.T + 2 * psf.kxy);
    const long long total = (long long)n * tl.tpp;
    const int Cmax = (tl.T + 4 * psf.kxy) * (tl.T + 4 * psf.kxy);   // padded coefficient array
    const size_t smem = (size_t)(2 * Lmax + Cmax) * sizeof(float);
    const bool fast = psf.kxy == 1 && psf.kz == 3;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (fast) {
        if ((e = prep(k_pose_vjp<1, 3, PlainVol>, smem)) != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pose_vjp<1, 3, PlainVol>, 256, smem);
    } else {
        if ((e = prep(k_pose_vjp<-1, -1, PlainVol>, smem)) != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pose_vjp<-1, -1, PlainVol>, 256, smem);
    }
    if (e != cudaSuccess) return e;
    long long grid = (long long)(per_sm > 0 ? per_sm : 1) * nsm;
    if (grid > total) grid = total;
    const long long slots = gbuf_tiles * Lmax / slot_stride(Lmax);   // padded slots in the scratch
    if (grid > slots) grid = slots;
    if (grid <= 0) return cudaErrorInvalidValue;
    if ((e = cudaMemsetAsync(counter, 0, sizeof(int), st)) != cudaSuccess) return e;
    if (fast)
        k_pose_vjp<1, 3, PlainVol><<<(unsigned)grid, 256, smem, st>>>(x, vd, desc, fix, psf, tl, total, r,
                                                                     gpart, gbuf, Lmax, counter);
    else
        k_pose_vjp<-1, -1, PlainVol><<<(unsigned)grid, 256, smem, st>>>(x, vd, desc, fix, psf, tl, total, r,
                                                                       gpart, gbuf, Lmax, counter);
    return cudaGetLastError();
}

// Tiles of gradient scratch needed per chunk (float planes of the lattice).
size_t ncc_gbuf_floats_per_tile(const Tiling &tl, int kxy)
{
    return 6 * (size_t)(tl.T + 2 * kxy) * (tl.T + 2 * kxy);
}

int ncc_launch_count(const Tiling &tl, int n, bool grad, long long gbuf_tiles)
{
    if (n <= 0) return 0;
    if (!grad) return 1;
    if (tl.tpp == 1) return 1;
    const long long total = (long long)n * tl.tpp, chunk = (gbuf_tiles / tl.tpp) * tl.tpp;
    return chunk > 0 ? (int)(2 * ((total + chunk - 1) / chunk)) : 0;
}

cudaError_t launch_ncc_finish(const DevGeom *g, const int32_t *desc, const double *poses, int n_params,
                              int n, const Tiling &tl, const double *part, const double *gpart,
                              int min_valid, double *ncc, double *grad, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_ncc_finish<<<(n + 127) / 128, 128, 0, st>>>(g, n_params, n, tl.tpp, desc, poses, part, gpart,
                                                  min_valid, ncc, grad);
    return cudaGetLastError();
}

}  // namespace pvr
