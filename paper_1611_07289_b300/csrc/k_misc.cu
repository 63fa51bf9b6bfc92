// Patch table construction (Sec. II "Patch Extraction"), patch pixel
// gather, and the evaluation metrics of Sec. IV-A.
#include <math.h>

#include <vector>

#include "pvr_internal.h"

namespace pvr {
namespace {

// Monotone map float -> unsigned so that unsigned max = float max.
__device__ __forceinline__ unsigned float_key(float f)
{
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_float(unsigned k)
{
    unsigned u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

__global__ void k_stack_max(const float *__restrict__ s, long long total, unsigned *__restrict__ out)
{
    __shared__ unsigned sh[32];
    unsigned m = 0u;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        m = max(m, float_key(s[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, sh[w]);
        atomicMax(out, m);
    }
}

// Candidate patches of one slice: corners (ix * stride, iy * stride) for
// ix < ncx, iy < ncy; candidates of all slices are numbered consecutively
// from cand_off.  The table has one entry per slice (over all stacks in
// order) plus a sentinel whose cand_off is the candidate count.
struct SliceCand {
    long long cand_off;
    int s, k, a, stride, ncx, ncy;
};

// Slice entry of candidate c (binary search over the cand_off prefix).
__device__ __forceinline__ const SliceCand &slice_of(const SliceCand *__restrict__ sc, int n_slices,
                                                     long long c)
{
    int lo = 0, hi = n_slices - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (sc[mid].cand_off <= c) lo = mid;
        else hi = mid - 1;
    }
    return sc[lo];
}

// One CTA per candidate patch: keep iff #pixels > fg level >= keep_frac a^2.
__global__ void __launch_bounds__(256) k_patch_keep(const DevGeom *__restrict__ g,
                                                    const float *__restrict__ stacks,
                                                    const SliceCand *__restrict__ sc, int n_slices,
                                                    double fg_frac, double keep_frac,
                                                    const unsigned *__restrict__ imax_key,
                                                    int32_t *__restrict__ keep)
{
    const long long c = blockIdx.x;
    const SliceCand e = slice_of(sc, n_slices, c);
    const int r = (int)(c - e.cand_off), a = e.a;
    const int y0 = (r / e.ncx) * e.stride, x0 = (r % e.ncx) * e.stride;
    const int W = g->sw[e.s], H = g->sh[e.s];
    const float *base = stacks + g->stack_off[e.s] + ((size_t)e.k * H + y0) * W + x0;
    const float thr = __fmul_rn((float)fg_frac, key_float(*imax_key));
    int cnt = 0;
    for (int t = threadIdx.x; t < a * a; t += blockDim.x) cnt += base[(size_t)(t / a) * W + t % a] > thr;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    __shared__ int sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
        keep[c] = (double)tot >= __dmul_rn(__dmul_rn(keep_frac, (double)a), (double)a) ? 1 : 0;
    }
}

// Single-CTA ordered compaction of the kept candidates into the table, with
// packed pixel offsets (exclusive prefix of a^2 over the kept candidates).
// counts[0] = kept patches; counts[1..2] = total pixels (int64, split).
__global__ void __launch_bounds__(1024) k_patch_compact(const int32_t *__restrict__ keep,
                                                        long long n_cand,
                                                        const SliceCand *__restrict__ sc,
                                                        int n_slices, int32_t *__restrict__ desc,
                                                        int max_out, int32_t *__restrict__ counts)
{
    __shared__ int warp_tot[32];
    __shared__ long long warp_pix[32];
    __shared__ long long base_sh, pix_sh;
    if (threadIdx.x == 0) base_sh = pix_sh = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (long long c0 = 0; c0 < n_cand; c0 += blockDim.x) {
        const long long c = c0 + threadIdx.x;
        const int f = (c < n_cand) ? keep[c] : 0;
        SliceCand e;
        e.a = 0;
        if (f) e = slice_of(sc, n_slices, c);
        const long long sz = f ? (long long)e.a * e.a : 0;
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
        if (f && idx < max_out) {
            const int r = (int)(c - e.cand_off);
            int32_t *d = desc + 8 * (size_t)idx;
            d[0] = e.s;
            d[1] = e.k;
            d[2] = (r % e.ncx) * e.stride;
            d[3] = (r / e.ncx) * e.stride;
            d[4] = e.a;
            d[5] = e.a;
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

__global__ void __launch_bounds__(256) k_patch_gather(const DevGeom *__restrict__ g,
                                                      const float *__restrict__ stacks,
                                                      const int32_t *__restrict__ desc,
                                                      long long n_pix, int32_t *__restrict__ err,
                                                      float *__restrict__ y)
{
    const int32_t *d = desc + 8 * (size_t)blockIdx.x;
    int s = d[0], k = d[1], x0 = d[2], y0 = d[3], w = d[4], h = d[5], off = d[6];
    if (s < 0 || s >= g->n_stacks || k < 0 || k >= g->sk[s] || x0 < 0 || y0 < 0 || w < 1 ||
        h < 1 || x0 + w > g->sw[s] || y0 + h > g->sh[s] || off < 0 ||
        (long long)off + (long long)w * h > n_pix) {
        if (threadIdx.x == 0) atomicOr(err, 1);
        return;
    }
    int W = g->sw[s], H = g->sh[s];
    const float *base = stacks + g->stack_off[s] + ((size_t)k * H + y0) * W + x0;
    float *dst = y + d[6];
    for (int t = threadIdx.x; t < w * h; t += blockDim.x) dst[t] = base[(size_t)(t / w) * W + t % w];
}

// ---------------------------------------------------------------- metrics --

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide max of a float (result in every thread); sh: 32 floats.
__device__ float block_max(float v, float *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    float m = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, sh[w]);
    __syncthreads();
    return m;
}

template <int NV>
__device__ void block_sums(double *v, double *sh)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < NV; ++k) v[k] = wsum(v[k]);
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < NV; ++k) sh[wid * NV + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[w * NV + k];
            v[k] = s;
        }
}

// pass 1: count, sum ref, sum img, max ref, min ref per block
__global__ void __launch_bounds__(256) k_metrics1(const float *__restrict__ ref,
                                                  const float *__restrict__ img,
                                                  const uint8_t *__restrict__ mask, long long n,
                                                  double *__restrict__ scr)
{
    __shared__ double sh[32 * 3];
    __shared__ float mx[32], mn[32];
    double v[3] = {0.0, 0.0, 0.0};
    float a = -INFINITY, b = INFINITY;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (mask && !mask[i]) continue;
        float r = ref[i];
        v[0] += 1.0;
        v[1] += r;
        v[2] += img[i];
        a = fmaxf(a, r);
        b = fminf(b, r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fminf(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if ((threadIdx.x & 31) == 0) {
        mx[threadIdx.x >> 5] = a;
        mn[threadIdx.x >> 5] = b;
    }
    block_sums<3>(v, sh);
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            a = fmaxf(a, mx[w]);
            b = fminf(b, mn[w]);
        }
        double *o = scr + 8 * (size_t)blockIdx.x;
        o[0] = v[0];
        o[1] = v[1];
        o[2] = v[2];
        o[3] = a;
        o[4] = b;
    }
}

// pass 2: centred sums with the means of pass 1 (folded here per block)
__global__ void __launch_bounds__(256) k_metrics2(const float *__restrict__ ref,
                                                  const float *__restrict__ img,
                                                  const uint8_t *__restrict__ mask, long long n,
                                                  const double *__restrict__ scr1, int nb,
                                                  double *__restrict__ scr2)
{
    __shared__ double sh[32 * 4];
    __shared__ double means[2];
    if (threadIdx.x == 0) {
        double c = 0, sr = 0, si = 0;
        for (int b = 0; b < nb; ++b) {
            c += scr1[8 * b];
            sr += scr1[8 * b + 1];
            si += scr1[8 * b + 2];
        }
        means[0] = c > 0 ? sr / c : 0.0;
        means[1] = c > 0 ? si / c : 0.0;
    }
    __syncthreads();
    const double mr = means[0], mi = means[1];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (mask && !mask[i]) continue;
        double a = (double)ref[i] - mr, b = (double)img[i] - mi, d = (double)img[i] - (double)ref[i];
        v[0] += a * a;
        v[1] += b * b;
        v[2] += a * b;
        v[3] += d * d;
    }
    block_sums<4>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) scr2[8 * (size_t)blockIdx.x + k] = v[k];
}

__global__ void k_metrics3(const double *__restrict__ scr1, const double *__restrict__ scr2, int nb,
                           double *__restrict__ out)
{
    double c = 0, sr = 0, si = 0, rmax = -INFINITY, rmin = INFINITY, vr = 0, vi = 0, cv = 0, se = 0;
    for (int b = 0; b < nb; ++b) {
        c += scr1[8 * b];
        sr += scr1[8 * b + 1];
        si += scr1[8 * b + 2];
        if (scr1[8 * b] > 0) {
            rmax = fmax(rmax, scr1[8 * b + 3]);
            rmin = fmin(rmin, scr1[8 * b + 4]);
        }
        vr += scr2[8 * b];
        vi += scr2[8 * b + 1];
        cv += scr2[8 * b + 2];
        se += scr2[8 * b + 3];
    }
    for (int k = 0; k < 5; ++k) out[k] = 0.0;
    if (c == 0) return;
    double mr = sr / c, mi = si / c;
    vr /= c;
    vi /= c;
    cv /= c;
    double mse = se / c;
    out[0] = mse > 0 ? 10.0 * log10(rmax * rmax / mse) : INFINITY;
    out[1] = (vr > 0 && vi > 0) ? cv / sqrt(vr * vi) : 0.0;
    double L = rmax - rmin, c1 = (0.01 * L) * (0.01 * L), c2 = (0.03 * L) * (0.03 * L);
    double ssim = ((2 * mr * mi + c1) * (2 * cv + c2)) / ((mr * mr + mi * mi + c1) * (vr + vi + c2));
    out[2] = ssim;
    out[3] = (1.0 - ssim) / 2.0;
    out[4] = mse;
}

// Per-patch evaluation, one CTA per patch: global PSNR, CC, SSIM, DSSIM of the
// simulated against the acquired patch over valid pixels (float64 sums), then
// the local SSIM of every valid pixel over the valid pixels of its
// (2w+1)^2 window clipped to the patch (same c1, c2), written as the DSSIM
// heat map, and the mean local SSIM.
// Local SSIM of pixel (i, j) from its window sums {k, sum a, sum b, sum a^2,
// sum b^2, sum ab} over the valid pixels of the window.
__device__ __forceinline__ double local_ssim(const double S[6], double c1, double c2)
{
    const double rk = 1.0 / S[0], ma = S[1] * rk, mb = S[2] * rk;   // one float64 division
    const double va = fmax(S[3] * rk - ma * ma, 0.0), vb = fmax(S[4] * rk - mb * mb, 0.0);
    const double cab = S[5] * rk - ma * mb;
    return ((2.0 * ma * mb + c1) * (2.0 * cab + c2)) / ((ma * ma + mb * mb + c1) * (va + vb + c2));
}

// Pass 3 with the window sums built row by row: row r of the patch is staged
// in shared memory, thread i forms its column's horizontal window sums R(i, r)
// (6 channels) into a ring of the 2w+1 rows of the current window, and the
// window sums of output row j are the ring's rows added in row order.  Every
// float64 product is formed once per (pixel, column of its window) instead of
// once per (pixel, window pixel).  wmax: patch width the ring is sized for.
__device__ void local_ssim_rows(const float *__restrict__ y, const float *__restrict__ sim,
                                const uint8_t *__restrict__ valid, size_t off, int W, int H, int w,
                                int wmax, double c1, double c2, float *__restrict__ map, double ls[2],
                                double *ring)
{
    const int nslot = 2 * w + 1;
    float *ry = reinterpret_cast<float *>(ring + (size_t)nslot * wmax * 6);
    float *rs = ry + wmax;
    uint8_t *rv = reinterpret_cast<uint8_t *>(rs + wmax);
    const int i = threadIdx.x;
    auto add_row = [&](int r) {   // stage row r and store its horizontal sums in slot r mod nslot
        __syncthreads();          // the previous row's staging is no longer read
        for (int t = threadIdx.x; t < W; t += blockDim.x) {
            const size_t q = off + (size_t)r * W + t;
            ry[t] = y[q];
            rs[t] = sim[q];
            rv[t] = valid[q];
        }
        __syncthreads();
        if (i < W) {
            double R[6] = {0, 0, 0, 0, 0, 0};
            for (int ii = max(i - w, 0); ii <= min(i + w, W - 1); ++ii) {
                if (!rv[ii]) continue;
                const double a = ry[ii], b = rs[ii];
                R[0] += 1.0;
                R[1] += a;
                R[2] += b;
                R[3] += a * a;
                R[4] += b * b;
                R[5] += a * b;
            }
            double *slot = ring + ((size_t)(r % nslot) * wmax + i) * 6;
#pragma unroll
            for (int c = 0; c < 6; ++c) slot[c] = R[c];
        }
    };
    for (int r = 0; r < min(w, H); ++r) add_row(r);
    for (int j = 0; j < H; ++j) {
        if (j + w < H) add_row(j + w);
        // the ring rows are this thread's own column: no barrier needed to read them
        if (i < W) {
            const size_t o = off + (size_t)j * W + i;
            if (!valid[o]) {
                if (map) map[o] = 0.f;
                continue;
            }
            double S[6] = {0, 0, 0, 0, 0, 0};
            for (int jj = max(j - w, 0); jj <= min(j + w, H - 1); ++jj) {
                const double *slot = ring + ((size_t)(jj % nslot) * wmax + i) * 6;
#pragma unroll
                for (int c = 0; c < 6; ++c) S[c] += slot[c];
            }
            const double ss = local_ssim(S, c1, c2);
            if (map) map[o] = (float)((1.0 - ss) / 2.0);
            ls[0] += ss;
            ls[1] += 1.0;
        }
    }
}

// wmax > 0: the ring of local_ssim_rows (dynamic shared memory) serves
// patches up to wmax pixels wide; wider ones, and wmax = 0, take the direct
// window loop.
__global__ void __launch_bounds__(256) k_patch_metrics(const float *__restrict__ y,
                                                       const float *__restrict__ sim,
                                                       const uint8_t *__restrict__ valid,
                                                       const int32_t *__restrict__ desc, int w,
                                                       double *__restrict__ out,
                                                       float *__restrict__ map, int wmax)
{
    extern __shared__ double ring[];
    __shared__ double sh[32 * 8];
    __shared__ double glob[8];
    const int32_t *d = desc + 8 * (size_t)blockIdx.x;
    const int W = d[4], H = d[5];
    const size_t off = (size_t)d[6];
    const int n = W * H;
    // pass 1: counts, sums, extremes of the acquired patch
    double v[5] = {0, 0, 0, 0, 0};
    float rmax = -INFINITY, rmin = INFINITY;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        if (!valid[off + t]) continue;
        const double a = y[off + t], b = sim[off + t];
        v[0] += 1.0;
        v[1] += a;
        v[2] += b;
        rmax = fmaxf(rmax, y[off + t]);
        rmin = fminf(rmin, y[off + t]);
    }
    block_sums<3>(v, sh);
    rmax = block_max(rmax, (float *)(sh + 32 * 4));
    rmin = -block_max(-rmin, (float *)(sh + 32 * 4));
    if (threadIdx.x == 0) {
        glob[0] = v[0];
        glob[1] = v[0] > 0.0 ? v[1] / v[0] : 0.0;
        glob[2] = v[0] > 0.0 ? v[2] / v[0] : 0.0;
        glob[3] = rmax;
        glob[4] = rmin;
    }
    __syncthreads();
    const double cnt = glob[0], mr = glob[1], mi = glob[2];
    // pass 2: centred second moments and squared error
    double u[4] = {0, 0, 0, 0};
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        if (!valid[off + t]) continue;
        const double a = (double)y[off + t] - mr, b = (double)sim[off + t] - mi;
        const double dd = (double)sim[off + t] - (double)y[off + t];
        u[0] += a * a;
        u[1] += b * b;
        u[2] += a * b;
        u[3] += dd * dd;
    }
    block_sums<4>(u, sh);
    const double L = glob[3] - glob[4];
    const double c1 = (0.01 * L) * (0.01 * L), c2 = (0.03 * L) * (0.03 * L);
    double *o = out + 5 * (size_t)blockIdx.x;
    if (threadIdx.x == 0) {
        if (cnt > 0.0) {
            const double vr = u[0] / cnt, vi = u[1] / cnt, cv = u[2] / cnt, mse = u[3] / cnt;
            o[0] = mse > 0.0 ? 10.0 * log10(glob[3] * glob[3] / mse) : INFINITY;
            o[1] = (vr > 0.0 && vi > 0.0) ? cv / sqrt(vr * vi) : 0.0;
            const double ss = ((2.0 * mr * mi + c1) * (2.0 * cv + c2)) / ((mr * mr + mi * mi + c1) * (vr + vi + c2));
            o[2] = ss;
            o[3] = (1.0 - ss) / 2.0;
        } else {
            o[0] = o[1] = o[2] = o[3] = 0.0;
        }
    }
    // pass 3: local SSIM map
    double ls[2] = {0.0, 0.0};
    if (W <= wmax && W <= (int)blockDim.x) {
        local_ssim_rows(y, sim, valid, off, W, H, w, wmax, c1, c2, map, ls, ring);
        block_sums<2>(ls, sh);
        if (threadIdx.x == 0) o[4] = ls[1] > 0.0 ? ls[0] / ls[1] : 0.0;
        return;
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int j = t / W, i = t - j * W;
        if (!valid[off + t]) {
            if (map) map[off + t] = 0.f;
            continue;
        }
        double k = 0.0, sa = 0.0, sb = 0.0, saa = 0.0, sbb = 0.0, sab = 0.0;
        for (int jj = max(j - w, 0); jj <= min(j + w, H - 1); ++jj)
            for (int ii = max(i - w, 0); ii <= min(i + w, W - 1); ++ii) {
                const size_t q = off + (size_t)jj * W + ii;
                if (!valid[q]) continue;
                const double a = y[q], b = sim[q];
                k += 1.0;
                sa += a;
                sb += b;
                saa += a * a;
                sbb += b * b;
                sab += a * b;
            }
        const double ma = sa / k, mb = sb / k;
        const double va = fmax(saa / k - ma * ma, 0.0), vb = fmax(sbb / k - mb * mb, 0.0);
        const double cab = sab / k - ma * mb;
        const double ss = ((2.0 * ma * mb + c1) * (2.0 * cab + c2)) / ((ma * ma + mb * mb + c1) * (va + vb + c2));
        if (map) map[off + t] = (float)((1.0 - ss) / 2.0);
        ls[0] += ss;
        ls[1] += 1.0;
    }
    block_sums<2>(ls, sh);
    if (threadIdx.x == 0) o[4] = ls[1] > 0.0 ? ls[0] / ls[1] : 0.0;
}

}  // namespace

constexpr int kMetricBlocks = 296;

cudaError_t launch_patches_build(const DevGeom *g, const pvr_geometry &hg, const float *stacks,
                                 int64_t total, const int32_t *slice_a, const int32_t *slice_stride,
                                 double fg_frac, double keep_frac, int32_t *desc_out, int max_out,
                                 int32_t *keep, int64_t *n_cand_out, unsigned *imax_key,
                                 int32_t *counts, void *slice_scratch, cudaStream_t st)
{
    std::vector<SliceCand> sc;
    long long nc = 0;
    int gk = 0;
    for (int s = 0; s < hg.n_stacks; ++s) {
        const int W = hg.stack_w[s], H = hg.stack_h[s];
        for (int k = 0; k < hg.stack_k[s]; ++k, ++gk) {
            SliceCand e;
            e.cand_off = nc;
            e.s = s;
            e.k = k;
            e.a = slice_a[gk];
            e.stride = slice_stride[gk];
            e.ncx = W >= e.a ? (W - e.a) / e.stride + 1 : 0;
            e.ncy = H >= e.a ? (H - e.a) / e.stride + 1 : 0;
            nc += (long long)e.ncx * e.ncy;
            sc.push_back(e);
        }
    }
    *n_cand_out = nc;
    const int n_slices = (int)sc.size();
    SliceCand *d_sc = (SliceCand *)slice_scratch;
    cudaError_t e;
    // from pageable memory: returns once the host vector has been staged
    if ((e = cudaMemcpyAsync(d_sc, sc.data(), sc.size() * sizeof(SliceCand), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess)
        return e;
    cudaMemsetAsync(imax_key, 0, sizeof(unsigned), st);
    cudaMemsetAsync(counts, 0, 4 * sizeof(int32_t), st);
    if (total > 0) k_stack_max<<<296, 256, 0, st>>>(stacks, (long long)total, imax_key);
    if (nc > 0) {
        k_patch_keep<<<(unsigned)nc, 256, 0, st>>>(g, stacks, d_sc, n_slices, fg_frac, keep_frac,
                                                   imax_key, keep);
        k_patch_compact<<<1, 1024, 0, st>>>(keep, nc, d_sc, n_slices, desc_out, max_out, counts);
    }
    return cudaGetLastError();
}

size_t patches_slice_scratch_bytes(int n_slices)
{
    return (size_t)(n_slices + 1) * sizeof(SliceCand);
}

cudaError_t launch_stack_max(const float *stacks, int64_t total, unsigned *imax_key, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(imax_key, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    if (total > 0) k_stack_max<<<296, 256, 0, st>>>(stacks, (long long)total, imax_key);
    return cudaGetLastError();
}

cudaError_t launch_patches_gather(const DevGeom *g, const float *stacks, const int32_t *desc,
                                  int n, int64_t n_pix, int32_t *err, float *y, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_patch_gather<<<(unsigned)n, 256, 0, st>>>(g, stacks, desc, (long long)n_pix, err, y);
    return cudaGetLastError();
}

cudaError_t launch_patch_metrics(const float *y, const float *sim, const uint8_t *valid, const int32_t *desc,
                                 int n, int w, int max_side, double *out, float *map, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    // the row ring (2w+1 rows of 6 float64 per column, plus one staged row)
    // when it fits 100 KB of shared memory; else the direct window loop
    int wmax = max_side <= 256 ? max_side : 0;
    size_t smem = wmax > 0 ? (size_t)(2 * w + 1) * wmax * 6 * sizeof(double) + (size_t)wmax * 9 + 16 : 0;
    if (smem > 100 * 1024) {
        wmax = 0;
        smem = 0;
    }
    cudaError_t e;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_patch_metrics, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
        return e;
    k_patch_metrics<<<(unsigned)n, 256, smem, st>>>(y, sim, valid, desc, w, out, map, wmax);
    return cudaGetLastError();
}

cudaError_t launch_metrics(const float *ref, const float *img, const uint8_t *mask, int64_t n,
                           double *scratch, double *out, cudaStream_t st)
{
    double *s1 = scratch, *s2 = scratch + 8 * kMetricBlocks;
    k_metrics1<<<kMetricBlocks, 256, 0, st>>>(ref, img, mask, (long long)n, s1);
    k_metrics2<<<kMetricBlocks, 256, 0, st>>>(ref, img, mask, (long long)n, s1, kMetricBlocks, s2);
    k_metrics3<<<1, 1, 0, st>>>(s1, s2, kMetricBlocks, out);
    return cudaGetLastError();
}

}  // namespace pvr
