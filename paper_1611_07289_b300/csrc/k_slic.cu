// Superpixel patches (Sec. II "Patch Extraction": SLIC superpixels,
// dilated by gamma pixels): simple linear iterative clustering on every
// slice of every stack, then one patch per superpixel -- the bounding box of
// the dilated superpixel with a membership mask.
//
// Readings where the paper is silent: centres start on a regular grid of
// nx = max(1, round(W / a)) columns of width sx = W / nx (likewise rows) at
// the cell centres with the intensity of the pixel under them; a pixel in
// grid cell (floor(x / sx), floor(y / sy)) compares the centres of the 3 x 3
// neighbouring cells by D^2 = dI^2 + (dx^2 + dy^2) (t / a)^2 in float32
// (each operation rounded, no contraction), ties to the lower centre index;
// centres move to the mean of their pixels (positions summed exactly as
// integers, intensities as round(1024 I)), a centre without pixels stays;
// no connectivity step.  Dilation: square structuring element of radius
// gamma.  A superpixel becomes a patch when its dilated box fits max_side
// (at most 128) and at least keep_frac of its member pixels exceed
// fg_frac * I_max.
#include <math.h>

#include <vector>

#include <algorithm>

#include "pvr_internal.h"

namespace pvr {
namespace {

struct SlicSlice {
    long long pix_off;   // first pixel of the slice in the packed stacks
    int s, k, W, H, nx, ny, c_off;
    double sx, sy;
};

constexpr int kSlicMaxBox = 128;

__device__ __forceinline__ int slice_of_pixel(const SlicSlice *__restrict__ sl, int n, long long p)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (sl[mid].pix_off <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_slic_init(const float *__restrict__ st, const SlicSlice *__restrict__ sl, int n_slices,
                            const int *__restrict__ c_slice, int C, float *__restrict__ cx,
                            float *__restrict__ cy, float *__restrict__ ci)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const SlicSlice e = sl[c_slice[c]];
    const int local = c - e.c_off, i = local % e.nx, j = local / e.nx;
    const float x = (float)(((double)i + 0.5) * e.sx), y = (float)(((double)j + 0.5) * e.sy);
    cx[c] = x;
    cy[c] = y;
    const int px = min((int)x, e.W - 1), py = min((int)y, e.H - 1);
    ci[c] = st[e.pix_off + (long long)py * e.W + px];
}

// Assignment of every stack pixel to its nearest centre, and the sums of the
// next update.
__global__ void k_slic_assign(const float *__restrict__ st, long long total, const SlicSlice *__restrict__ sl,
                              int n_slices, const float *__restrict__ cx, const float *__restrict__ cy,
                              const float *__restrict__ ci, float m2, int32_t *__restrict__ label,
                              int *__restrict__ cnt, unsigned long long *__restrict__ sums)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const SlicSlice e = sl[slice_of_pixel(sl, n_slices, p)];
        const int r = (int)(p - e.pix_off), y = r / e.W, x = r - y * e.W;
        const float I = st[p], xf = (float)x, yf = (float)y;
        const int gx = min((int)floor((double)x / e.sx), e.nx - 1), gy = min((int)floor((double)y / e.sy), e.ny - 1);
        float best = INFINITY;
        int lab = 0x7fffffff;
        for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
                const int cj = gy + dj, cii = gx + di;
                if (cj < 0 || cj >= e.ny || cii < 0 || cii >= e.nx) continue;
                const int c = e.c_off + cj * e.nx + cii;
                const float dI = __fsub_rn(I, ci[c]), dx = __fsub_rn(xf, cx[c]), dy = __fsub_rn(yf, cy[c]);
                const float d = __fadd_rn(__fmul_rn(dI, dI),
                                          __fmul_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), m2));
                if (d < best || (d == best && c < lab)) {
                    best = d;
                    lab = c;
                }
            }
        label[p] = lab;
        atomicAdd(cnt + lab, 1);
        atomicAdd(sums + 3 * (size_t)lab, (unsigned long long)x);
        atomicAdd(sums + 3 * (size_t)lab + 1, (unsigned long long)y);
        atomicAdd(sums + 3 * (size_t)lab + 2, (unsigned long long)llrint((double)I * 1024.0));
    }
}

__global__ void k_slic_update(int C, int *__restrict__ cnt, unsigned long long *__restrict__ sums,
                              float *__restrict__ cx, float *__restrict__ cy, float *__restrict__ ci)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int n = cnt[c];
    if (n > 0) {
        cx[c] = (float)((double)(long long)sums[3 * (size_t)c] / n);
        cy[c] = (float)((double)(long long)sums[3 * (size_t)c + 1] / n);
        ci[c] = (float)((double)(long long)sums[3 * (size_t)c + 2] / 1024.0 / n);
    }
    cnt[c] = 0;
    sums[3 * (size_t)c] = sums[3 * (size_t)c + 1] = sums[3 * (size_t)c + 2] = 0ull;
}

__global__ void k_slic_bbox(long long total, const SlicSlice *__restrict__ sl, int n_slices,
                            const int32_t *__restrict__ label, int *__restrict__ box)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const SlicSlice e = sl[slice_of_pixel(sl, n_slices, p)];
        const int r = (int)(p - e.pix_off), y = r / e.W, x = r - y * e.W, c = label[p];
        atomicMin(box + 4 * (size_t)c, x);
        atomicMax(box + 4 * (size_t)c + 1, x);
        atomicMin(box + 4 * (size_t)c + 2, y);
        atomicMax(box + 4 * (size_t)c + 3, y);
    }
}

// Dilated membership of centre c over its dilated box (w x h, origin x0, y0)
// in shared memory: eq = (label == c), then the square dilation as a
// horizontal and a vertical running count (one thread per row / column).
__device__ void dilate_box(const int32_t *__restrict__ label, const SlicSlice &e, int c, int x0, int y0, int w, int h,
                           int gamma, uint8_t *eq, uint8_t *hor)
{
    for (int t = threadIdx.x; t < w * h; t += blockDim.x) {
        const int yy = t / w, xx = t - yy * w;
        eq[t] = label[e.pix_off + (long long)(y0 + yy) * e.W + (x0 + xx)] == c;
    }
    __syncthreads();
    for (int yy = threadIdx.x; yy < h; yy += blockDim.x) {
        int run = 0;
        for (int xx = 0; xx < min(gamma, w); ++xx) run += eq[yy * w + xx];
        for (int xx = 0; xx < w; ++xx) {
            if (xx + gamma < w) run += eq[yy * w + xx + gamma];
            if (xx - gamma - 1 >= 0) run -= eq[yy * w + xx - gamma - 1];
            hor[yy * w + xx] = run > 0;
        }
    }
    __syncthreads();
    for (int xx = threadIdx.x; xx < w; xx += blockDim.x) {
        int run = 0;
        for (int yy = 0; yy < min(gamma, h); ++yy) run += hor[yy * w + xx];
        for (int yy = 0; yy < h; ++yy) {
            if (yy + gamma < h) run += hor[(yy + gamma) * w + xx];
            if (yy - gamma - 1 >= 0) run -= hor[(yy - gamma - 1) * w + xx];
            eq[yy * w + xx] = run > 0;   // eq's own row values are no longer needed
        }
    }
    __syncthreads();
}

// Per centre: dilated box, membership count and foreground count: keep flag
// and the box (x0, y0, w, h) for the compaction.
__global__ void __launch_bounds__(256) k_slic_keep(const float *__restrict__ st, const SlicSlice *__restrict__ sl,
                                                   const int *__restrict__ c_slice, const int32_t *__restrict__ label,
                                                   const int *__restrict__ box, int gamma, int max_side,
                                                   double fg_frac, double keep_frac,
                                                   const unsigned *__restrict__ imax_key, int *__restrict__ keep,
                                                   int *__restrict__ geo)
{
    __shared__ uint8_t eq[kSlicMaxBox * kSlicMaxBox], hor[kSlicMaxBox * kSlicMaxBox];
    __shared__ int red[2][32];
    const int c = blockIdx.x;
    const SlicSlice e = sl[c_slice[c]];
    const int bx0 = box[4 * (size_t)c], bx1 = box[4 * (size_t)c + 1];
    const int by0 = box[4 * (size_t)c + 2], by1 = box[4 * (size_t)c + 3];
    const int x0 = max(bx0 - gamma, 0), x1 = min(bx1 + gamma, e.W - 1);
    const int y0 = max(by0 - gamma, 0), y1 = min(by1 + gamma, e.H - 1);
    const int w = x1 - x0 + 1, h = y1 - y0 + 1;
    if (bx0 > bx1 || w > max_side || h > max_side) {   // empty superpixel or box too large
        if (threadIdx.x == 0) keep[c] = 0;
        return;
    }
    dilate_box(label, e, c, x0, y0, w, h, gamma, eq, hor);
    const unsigned kk = *imax_key;
    const float imax = __uint_as_float((kk & 0x80000000u) ? (kk & 0x7fffffffu) : ~kk);
    const float thr = __fmul_rn((float)fg_frac, imax);
    int nm = 0, nf = 0;
    for (int t = threadIdx.x; t < w * h; t += blockDim.x) {
        if (!eq[t]) continue;
        const int yy = t / w, xx = t - yy * w;
        ++nm;
        nf += st[e.pix_off + (long long)(y0 + yy) * e.W + (x0 + xx)] > thr;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nm += __shfl_xor_sync(0xffffffffu, nm, o);
        nf += __shfl_xor_sync(0xffffffffu, nf, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = nm;
        red[1][threadIdx.x >> 5] = nf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0, b = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            a += red[0][k];
            b += red[1][k];
        }
        keep[c] = (double)b >= __dmul_rn(keep_frac, (double)a) ? 1 : 0;
        geo[4 * (size_t)c] = x0;
        geo[4 * (size_t)c + 1] = y0;
        geo[4 * (size_t)c + 2] = w;
        geo[4 * (size_t)c + 3] = h;
    }
}

// Ordered compaction (single CTA): table rows in centre order with packed
// pixel offsets.  counts[0] = kept patches; counts[1..2] = pixels (int64).
__global__ void __launch_bounds__(1024) k_slic_compact(const int *__restrict__ keep, const int *__restrict__ geo,
                                                       const SlicSlice *__restrict__ sl,
                                                       const int *__restrict__ c_slice, int C,
                                                       int32_t *__restrict__ desc, int max_out,
                                                       int32_t *__restrict__ counts, int32_t *__restrict__ row_of)
{
    __shared__ int warp_tot[32];
    __shared__ long long warp_pix[32];
    __shared__ long long base_sh, pix_sh;
    if (threadIdx.x == 0) base_sh = pix_sh = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c0 = 0; c0 < C; c0 += blockDim.x) {
        const int c = c0 + threadIdx.x;
        const int f = c < C ? keep[c] : 0;
        const long long sz = f ? (long long)geo[4 * (size_t)c + 2] * geo[4 * (size_t)c + 3] : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        const int pre = __popc(bal & ((1u << lane) - 1u));
        long long v = sz;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) {
            warp_tot[wid] = __popc(bal);
            warp_pix[wid] = v;
        }
        __syncthreads();
        int woff = 0, tot = 0;
        long long poff = 0, ptot = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < wid) {
                woff += warp_tot[w];
                poff += warp_pix[w];
            }
            tot += warp_tot[w];
            ptot += warp_pix[w];
        }
        const long long idx = base_sh + woff + pre;
        if (c < C) row_of[c] = (f && idx < max_out) ? (int32_t)idx : -1;
        if (f && idx < max_out) {
            const SlicSlice e = sl[c_slice[c]];
            int32_t *d = desc + 8 * (size_t)idx;
            d[0] = e.s;
            d[1] = e.k;
            d[2] = geo[4 * (size_t)c];
            d[3] = geo[4 * (size_t)c + 1];
            d[4] = geo[4 * (size_t)c + 2];
            d[5] = geo[4 * (size_t)c + 3];
            d[6] = (int32_t)(pix_sh + poff + (v - sz));
            d[7] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            base_sh += tot;
            pix_sh += ptot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        counts[0] = (int32_t)base_sh;
        counts[1] = (int32_t)(pix_sh & 0xffffffffLL);
        counts[2] = (int32_t)(pix_sh >> 32);
    }
}

// Membership masks of the table rows (one CTA per centre that became a row).
__global__ void __launch_bounds__(256) k_slic_member(const SlicSlice *__restrict__ sl, const int *__restrict__ c_slice,
                                                     const int32_t *__restrict__ label, const int32_t *__restrict__ row_of,
                                                     const int32_t *__restrict__ desc, int gamma, long long max_pix,
                                                     uint8_t *__restrict__ member)
{
    __shared__ uint8_t eq[kSlicMaxBox * kSlicMaxBox], hor[kSlicMaxBox * kSlicMaxBox];
    const int c = blockIdx.x, row = row_of[c];
    if (row < 0) return;
    const SlicSlice e = sl[c_slice[c]];
    const int32_t *d = desc + 8 * (size_t)row;
    const int x0 = d[2], y0 = d[3], w = d[4], h = d[5];
    const long long off = d[6];
    if (off + (long long)w * h > max_pix) return;   // beyond the member buffer: left to the caller's check
    dilate_box(label, e, c, x0, y0, w, h, gamma, eq, hor);
    for (int t = threadIdx.x; t < w * h; t += blockDim.x) member[off + t] = eq[t];
}

}  // namespace

// Superpixel centres of every slice for superpixel size a: max(1, round(W/a))
// x max(1, round(H/a)) per slice (never more for a larger a).
int64_t slic_centres(const pvr_geometry &hg, int a)
{
    int64_t C = 0;
    for (int s = 0; s < hg.n_stacks; ++s) {
        const int64_t nx = std::max<int64_t>(1, lround((double)hg.stack_w[s] / a));
        const int64_t ny = std::max<int64_t>(1, lround((double)hg.stack_h[s] / a));
        C += (int64_t)hg.stack_k[s] * nx * ny;
    }
    return C;
}

namespace {

// Carving of the superpixel scratch: 256-byte aligned pieces.
struct SlicScratch {
    SlicSlice *sl;
    int *cs, *cnt, *box, *keep, *geo;
    int32_t *label, *row_of;
    float *cx, *cy, *ci;
    unsigned long long *sums;
};

size_t carve(void *base, int n_slices, int64_t C, int64_t total, SlicScratch *out)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        void *p = base ? (void *)((char *)base + off) : nullptr;
        off += (bytes + 255) / 256 * 256;
        return p;
    };
    SlicScratch s;
    s.sl = (SlicSlice *)take((size_t)n_slices * sizeof(SlicSlice));
    s.cs = (int *)take((size_t)C * sizeof(int));
    s.cnt = (int *)take((size_t)C * sizeof(int));
    s.box = (int *)take((size_t)C * 4 * sizeof(int));
    s.keep = (int *)take((size_t)C * sizeof(int));
    s.geo = (int *)take((size_t)C * 4 * sizeof(int));
    s.row_of = (int32_t *)take((size_t)C * sizeof(int32_t));
    s.label = (int32_t *)take((size_t)total * sizeof(int32_t));
    s.cx = (float *)take((size_t)C * sizeof(float));
    s.cy = (float *)take((size_t)C * sizeof(float));
    s.ci = (float *)take((size_t)C * sizeof(float));
    s.sums = (unsigned long long *)take((size_t)C * 3 * sizeof(unsigned long long));
    if (out) *out = s;
    return off;
}

}  // namespace

size_t slic_scratch_bytes(const pvr_geometry &hg, int a_min, int64_t total)
{
    int n_slices = 0;
    for (int s = 0; s < hg.n_stacks; ++s) n_slices += hg.stack_k[s];
    return carve(nullptr, n_slices, slic_centres(hg, a_min), total, nullptr);
}

cudaError_t launch_patches_build_slic(const DevGeom *g, const pvr_geometry &hg, const float *stacks, int64_t total,
                                      int a, double t, int gamma, int n_iter, double fg_frac, double keep_frac,
                                      int max_side, int32_t *desc_out, int max_out, uint8_t *member_out,
                                      int64_t max_pix, unsigned *imax_key, int32_t *counts, int64_t *n_centres_out,
                                      void *scratch, cudaStream_t st)
{
    (void)g;
    std::vector<SlicSlice> sl;
    std::vector<int> c_slice;
    long long off = 0;
    int C = 0;
    for (int s = 0; s < hg.n_stacks; ++s) {
        const int W = hg.stack_w[s], H = hg.stack_h[s];
        for (int k = 0; k < hg.stack_k[s]; ++k) {
            SlicSlice e;
            e.pix_off = off;
            e.s = s;
            e.k = k;
            e.W = W;
            e.H = H;
            e.nx = (int)lround((double)W / a);
            e.ny = (int)lround((double)H / a);
            if (e.nx < 1) e.nx = 1;
            if (e.ny < 1) e.ny = 1;
            e.sx = (double)W / e.nx;
            e.sy = (double)H / e.ny;
            e.c_off = C;
            for (int i = 0; i < e.nx * e.ny; ++i) c_slice.push_back((int)sl.size());
            C += e.nx * e.ny;
            sl.push_back(e);
            off += (long long)W * H;
        }
    }
    *n_centres_out = C;
    const int n_slices = (int)sl.size();
    // the context's superpixel scratch (sized for its smallest superpixel size)
    SlicScratch sc;
    carve(scratch, n_slices, C, total, &sc);
    SlicSlice *d_sl = sc.sl;
    int *d_cs = sc.cs, *cnt = sc.cnt, *box = sc.box, *keep = sc.keep, *geo = sc.geo;
    int32_t *label = sc.label, *row_of = sc.row_of;
    float *cx = sc.cx, *cy = sc.cy, *ci = sc.ci;
    unsigned long long *sums = sc.sums;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_sl, sl.data(), sl.size() * sizeof(SlicSlice), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_cs, c_slice.data(), c_slice.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, (size_t)C * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sums, 0, (size_t)C * 3 * sizeof(unsigned long long), st);
    if (e == cudaSuccess && C > 0) {
        const float m2 = (float)((t / a) * (t / a));
        k_slic_init<<<(C + 255) / 256, 256, 0, st>>>(stacks, d_sl, n_slices, d_cs, C, cx, cy, ci);
        for (int it = 0; it < n_iter; ++it) {
            k_slic_assign<<<1184, 256, 0, st>>>(stacks, (long long)total, d_sl, n_slices, cx, cy, ci, m2, label, cnt,
                                                sums);
            k_slic_update<<<(C + 255) / 256, 256, 0, st>>>(C, cnt, sums, cx, cy, ci);
        }
        // boxes: min x, max x, min y, max y (initialised empty)
        std::vector<int> binit((size_t)C * 4);
        for (int c = 0; c < C; ++c) {
            binit[4 * (size_t)c] = 0x7fffffff;
            binit[4 * (size_t)c + 1] = -1;
            binit[4 * (size_t)c + 2] = 0x7fffffff;
            binit[4 * (size_t)c + 3] = -1;
        }
        e = cudaMemcpyAsync(box, binit.data(), binit.size() * sizeof(int), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            k_slic_bbox<<<1184, 256, 0, st>>>((long long)total, d_sl, n_slices, label, box);
            k_slic_keep<<<C, 256, 0, st>>>(stacks, d_sl, d_cs, label, box, gamma, max_side, fg_frac, keep_frac,
                                           imax_key, keep, geo);
            k_slic_compact<<<1, 1024, 0, st>>>(keep, geo, d_sl, d_cs, C, desc_out, max_out, counts, row_of);
            k_slic_member<<<C, 256, 0, st>>>(d_sl, d_cs, label, row_of, desc_out, gamma, max_pix, member_out);
            e = cudaGetLastError();
        }
    }
    return e;
}

}  // namespace pvr
