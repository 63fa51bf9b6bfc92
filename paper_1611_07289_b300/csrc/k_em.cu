// EM robust statistics (Sec. II "EM-Based Outlier Removal", Eqs. m, p,
// p-bar), the weighted SIRT volume update and the per-patch registration
// optimiser step.
//
// Pixel work (residual statistics, E-step) runs on the same (patch, tile)
// grid as the forward model and leaves float64 partial sums per tile, so
// every reduction is deterministic: the partials are folded in a fixed order
// in float64 (the M-step and the patch-level model, whose stability needs
// it), by a single-CTA kernel or by the last block of the kernel that wrote
// them.
#include <math.h>

#include "pvr_internal.h"

namespace pvr {
namespace {

constexpr int kRedThreads = 1024;

// Pixel range of block's (patch, tile).
struct TileRange {
    int p, t, off, w, i0, j0, tw, th;
};

// Row of pixel pp of a tile tw pixels wide, from r = 1 / tw: (pp + 0.5) / tw
// lies at least 0.5 / tw from an integer and the two float roundings move it
// by less than that for pp < 2^22, so truncation gives floor(pp / tw).
__device__ __forceinline__ int tile_row(int pp, float r)
{
    return (int)(((float)pp + 0.5f) * r);
}

// Returns false for an empty tile or a descriptor whose pixel range is not
// inside [0, n_pix) (then err gets bit 1 and nothing is touched).
__device__ __forceinline__ bool tile_range(const int32_t *__restrict__ desc, const Tiling &tl,
                                           long long n_pix, int32_t *err, TileRange &r)
{
    r.p = blockIdx.x / tl.tpp;
    r.t = blockIdx.x % tl.tpp;
    const int32_t *d = desc + 8 * (size_t)r.p;
    r.w = d[4];
    int h = d[5];
    r.off = d[6];
    if (r.w < 1 || h < 1 || r.off < 0 || (long long)r.off + (long long)r.w * h > n_pix) {
        if (threadIdx.x == 0 && r.t == 0) atomicOr(err, 1);
        return false;
    }
    r.i0 = (r.t % tl.tiles_x) * tl.T;
    r.j0 = (r.t / tl.tiles_x) * tl.T;
    if (r.i0 >= r.w || r.j0 >= h) return false;
    r.tw = min(tl.T, r.w - r.i0);
    r.th = min(tl.T, h - r.j0);
    return true;
}

// Block sum / min / max of NV doubles; every thread gets the result.
template <int NV>
__device__ void block_reduce(double *v, double *sh, int op /*0 sum, 1 min, 2 max*/)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double y = __shfl_xor_sync(0xffffffffu, x, o);
            x = op == 0 ? x + y : (op == 1 ? fmin(x, y) : fmax(x, y));
        }
        v[k] = x;
    }
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < NV; ++k) sh[wid * NV + k] = v[k];
    __syncthreads();
    for (int k = 0; k < NV; ++k) {
        double x = sh[k];
        for (int w = 1; w < nw; ++w) {
            double y = sh[w * NV + k];
            x = op == 0 ? x + y : (op == 1 ? fmin(x, y) : fmax(x, y));
        }
        v[k] = x;
    }
    __syncthreads();
}

__device__ __forceinline__ double clampd(double v, double lo, double hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

// Residual statistics of a tile for a standalone EM call:
// part[0..3] = {N_valid, sum e^2, min e, max e}, e = y - sim (sim null: e = y).
__global__ void __launch_bounds__(256) k_em_stats(const float *__restrict__ y,
                                                  const float *__restrict__ sim,
                                                  const uint8_t *__restrict__ valid,
                                                  const int32_t *__restrict__ desc, Tiling tl,
                                                  long long n_pix, int32_t *__restrict__ err,
                                                  double *__restrict__ part)
{
    __shared__ double sh[32 * 2];
    TileRange r;
    double *pt = part + (size_t)blockIdx.x * kPartStride;
    if (!tile_range(desc, tl, n_pix, err, r)) {
        if (threadIdx.x < 4) pt[threadIdx.x] = 0.0;
        return;
    }
    double a[2] = {0.0, 0.0};
    double mn[1] = {INFINITY}, mx[1] = {-INFINITY};
    const float rtw = 1.0f / (float)r.tw;
    for (int pp = threadIdx.x; pp < r.tw * r.th; pp += blockDim.x) {
        const int row = tile_row(pp, rtw);
        size_t o = (size_t)r.off + (size_t)(r.j0 + row) * r.w + r.i0 + (pp - row * r.tw);
        if (!valid[o]) continue;
        float e = sim ? y[o] - sim[o] : y[o];
        a[0] += 1.0;
        a[1] += (double)(e * e);
        mn[0] = fmin(mn[0], (double)e);
        mx[0] = fmax(mx[0], (double)e);
    }
    block_reduce<2>(a, sh, 0);
    block_reduce<1>(mn, sh, 1);
    block_reduce<1>(mx, sh, 2);
    if (threadIdx.x == 0) {
        pt[0] = a[0];
        pt[1] = a[1];
        pt[2] = mn[0];
        pt[3] = mx[0];
    }
}

// Step 1-3: participating-pixel statistics -> initial sigma^2, c (first
// call), outlier density m, E-step constants.
// pstat: [0] sigma^2 floor, [1] first call, [2] m, [3] 1/(2 sigma^2),
//        [4] m (1-c) sqrt(2 pi) sigma / c.
__global__ void __launch_bounds__(kRedThreads) k_em_prepare(int n, int tpp,
                                                            const uint8_t *__restrict__ mask_in,
                                                            const double *__restrict__ part,
                                                            double *__restrict__ state,
                                                            double *__restrict__ pstat, double c0,
                                                            double floor_rel)
{
    __shared__ double sh[32 * 2];
    double a[2] = {0.0, 0.0}, mn[1] = {INFINITY}, mx[1] = {-INFINITY};
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        // the mask and the partials are loaded together (16-byte loads)
        const bool in = !mask_in || mask_in[p];
        for (int t = 0; t < tpp; ++t) {
            const double2 *pt = reinterpret_cast<const double2 *>(part + ((size_t)p * tpp + t) * kPartStride);
            const double2 u = pt[0], v = pt[1];   // {N, sum e^2}, {min e, max e}
            if (in && u.x > 0.0) {
                a[0] += u.x;
                a[1] += u.y;
                mn[0] = fmin(mn[0], v.x);
                mx[0] = fmax(mx[0], v.y);
            }
        }
    }
    block_reduce<2>(a, sh, 0);
    block_reduce<1>(mn, sh, 1);
    block_reduce<1>(mx, sh, 2);
    if (threadIdx.x == 0) {
        double npart = a[0];
        double range = npart > 0.0 ? mx[0] - mn[0] : 0.0;
        double sfloor = (floor_rel * range) * (floor_rel * range);
        if (sfloor < 1e-12) sfloor = 1e-12;
        bool first = state[PVR_ST_INIT] == 0.0;
        if (first) {
            double s2 = npart > 0.0 ? a[1] / npart : 1.0;
            state[PVR_ST_SIGMA2] = s2 < sfloor ? sfloor : s2;
            state[PVR_ST_C] = clampd(c0, 1e-3, 1.0 - 1e-3);
        }
        double m = range >= 1e-12 ? 1.0 / range : 0.0;
        double s2 = state[PVR_ST_SIGMA2], c = state[PVR_ST_C];
        state[PVR_ST_M] = m;
        state[PVR_ST_SIGMA2_USED] = s2;
        state[PVR_ST_EMIN] = mn[0];
        state[PVR_ST_EMAX] = mx[0];
        state[PVR_ST_N_PART] = npart;
        pstat[0] = sfloor;
        pstat[1] = first ? 1.0 : 0.0;
        pstat[2] = m;
        pstat[3] = 1.0 / (2.0 * s2);
        pstat[4] = m * (1.0 - c) * sqrt(2.0 * 3.14159265358979323846) * sqrt(s2) / c;
    }
}

// Step 4: E-step p = G c / (G c + m (1 - c)) = 1 / (1 + K exp(e^2 / 2 sigma^2)),
// K = m (1 - c) sqrt(2 pi) sigma / c; p = 1 if m = 0; p = 0 on invalid pixels.
// part[4..7] = {sum p, sum p e^2 (participating), sum p^2, N_valid}.
__global__ void __launch_bounds__(256) k_em_estep(const float *__restrict__ y,
                                                  const float *__restrict__ sim,
                                                  const uint8_t *__restrict__ valid,
                                                  const int32_t *__restrict__ desc, Tiling tl,
                                                  long long n_pix, int32_t *__restrict__ err,
                                                  const uint8_t *__restrict__ mask_in,
                                                  const double *__restrict__ pstat,
                                                  float *__restrict__ p_out,
                                                  double *__restrict__ part)
{
    __shared__ double sh[32 * 4];
    TileRange r;
    double *pt = part + (size_t)blockIdx.x * kPartStride;
    if (!tile_range(desc, tl, n_pix, err, r)) {
        if (threadIdx.x < 4) pt[4 + threadIdx.x] = 0.0;
        return;
    }
    const bool m_zero = pstat[2] == 0.0;
    const float inv2s2 = (float)pstat[3], K = (float)pstat[4];
    const bool part_in = !mask_in || mask_in[r.p];
    float sp = 0.f, spe2 = 0.f, sp2 = 0.f, nv = 0.f;
    auto pixel = [&](bool v, float e) {
        float pv = 0.f;
        if (v) {
            pv = m_zero ? 1.f : 1.f / (1.f + K * expf(e * e * inv2s2));
            if (part_in) {
                sp += pv;
                spe2 = fmaf(pv * e, e, spe2);
            }
            sp2 = fmaf(pv, pv, sp2);
            nv += 1.f;
        }
        return pv;
    };
    if (((r.off | r.w | r.i0 | r.tw) & 3) == 0) {
        // rows of whole 16-byte groups: four pixels per 16-byte load and store
        const int qw = r.tw >> 2;
        const float rqw = 1.0f / (float)qw;
        for (int qq = threadIdx.x; qq < qw * r.th; qq += blockDim.x) {
            const int row = tile_row(qq, rqw);
            const size_t o = (size_t)r.off + (size_t)(r.j0 + row) * r.w + r.i0 + 4 * (qq - row * qw);
            const uchar4 v = *reinterpret_cast<const uchar4 *>(valid + o);
            float4 e = *reinterpret_cast<const float4 *>(y + o);
            if (sim) {
                const float4 s4 = *reinterpret_cast<const float4 *>(sim + o);
                e.x -= s4.x;
                e.y -= s4.y;
                e.z -= s4.z;
                e.w -= s4.w;
            }
            float4 pv;
            pv.x = pixel(v.x, e.x);
            pv.y = pixel(v.y, e.y);
            pv.z = pixel(v.z, e.z);
            pv.w = pixel(v.w, e.w);
            *reinterpret_cast<float4 *>(p_out + o) = pv;
        }
    } else {
        const float rtw = 1.0f / (float)r.tw;
        for (int pp = threadIdx.x; pp < r.tw * r.th; pp += blockDim.x) {
            const int row = tile_row(pp, rtw);
            size_t o = (size_t)r.off + (size_t)(r.j0 + row) * r.w + r.i0 + (pp - row * r.tw);
            const bool v = valid[o];
            p_out[o] = pixel(v, v ? (sim ? y[o] - sim[o] : y[o]) : 0.f);
        }
    }
    // float32 tile sums (at most a 64 x 64 tile: counts exact, sums to ~1e-7)
    float a[4] = {sp, spe2, sp2, nv};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
    float *fs = reinterpret_cast<float *>(sh);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 4; ++k) fs[wid * 4 + k] = a[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) {
            float t = 0.f;
            for (int w = 0; w < nw; ++w) t += fs[w * 4 + k];
            pt[4 + k] = (double)t;
        }
}

// Steps 5-7: M-step, patch potentials and patch classification, spread over
// the grid (one thread per patch); the per-block partial sums are folded by
// the last block of each kernel (last_block) -- the patch-level model
// evaluates a float64 exponential per patch and EM iteration.
// pstat: [5] patch outlier density m_p, [6] stop flag of the patch EM loop,
// [7] number of eligible patches.  bpart: kEmBlockMax x 8 float64.
constexpr int kEmBlockMax = 512;

// Grid-wide fold without a second launch: every block publishes its
// partials, fences, and counts itself in; the block that arrives last (every
// partial visible after its own fence) does the fold and resets the counter
// for the next launch.  No block waits for another.
__device__ __forceinline__ bool last_block(unsigned *counter)
{
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(counter, 1u);
        s_last = prev == gridDim.x - 1;
        if (s_last) *counter = 0u;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

__device__ __forceinline__ void store_block(double *bpart, const double *v, int nv)
{
    if (threadIdx.x == 0)
        for (int k = 0; k < nv; ++k) bpart[(size_t)blockIdx.x * 8 + k] = v[k];
}

// Field k of the nb block partials folded by the 32 lanes of one warp in a
// fixed order (lane l takes blocks l, l + 32, ..., then a butterfly of
// shuffles, whose pairwise operations are commutative, so every lane holds
// the same value): the loads are issued together instead of one after the
// other by a single thread.  op: 0 sum, 1 min, 2 max.
__device__ __forceinline__ double warp_fold(int nb, const double *__restrict__ bpart, int k, int op)
{
    double s = op == 0 ? 0.0 : (op == 1 ? INFINITY : -INFINITY);
    for (int b = threadIdx.x & 31; b < nb; b += 32) {
        const double v = bpart[8 * (size_t)b + k];
        s = op == 0 ? s + v : (op == 1 ? fmin(s, v) : fmax(s, v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_xor_sync(0xffffffffu, s, o);
        s = op == 0 ? s + t : (op == 1 ? fmin(s, t) : fmax(s, t));
    }
    return s;
}

// Fold of k_em_patch_pot (called by the 32 lanes of warp 0 of the last
// block): pixel-level M-step, patch outlier density, first-call
// initialisation of the patch-level model.
__device__ void em_patch_head(int nb, const double *__restrict__ bpart, double *__restrict__ state,
                              double *__restrict__ pstat, double c0, int rule)
{
    const double sp = warp_fold(nb, bpart, 0, 0), spe2 = warp_fold(nb, bpart, 1, 0);
    const double ps = warp_fold(nb, bpart, 2, 0), ps2 = warp_fold(nb, bpart, 3, 0);
    const double ne = warp_fold(nb, bpart, 4, 0);
    const double mn = warp_fold(nb, bpart, 5, 1), mx = warp_fold(nb, bpart, 6, 2);
    if ((threadIdx.x & 31) != 0) return;
    double sfloor = pstat[0], npart = state[PVR_ST_N_PART];
    if (sp > 0.0) {
        double s2 = spe2 / sp;
        state[PVR_ST_SIGMA2] = s2 < sfloor ? sfloor : s2;
    }
    if (npart > 0.0) state[PVR_ST_C] = clampd(sp / npart, 1e-3, 1.0 - 1e-3);
    state[PVR_ST_SUM_P] = sp;
    state[PVR_ST_SUM_PE2] = spe2;
    double mp = (ne > 0.0 && mx - mn >= 1e-12) ? 1.0 / (mx - mn) : 0.0;
    pstat[5] = mp;
    pstat[6] = rule == 1 ? 1.0 : 0.0;
    pstat[7] = ne;
    if (rule == 0 && pstat[1] != 0.0) {
        double mu = ne > 0.0 ? ps / ne : 0.0;
        double var = ne > 0.0 ? ps2 / ne - mu * mu : 0.0;
        state[PVR_ST_MU_P] = mu;
        state[PVR_ST_SIGMA2_P] = var < 1e-4 ? 1e-4 : var;
        state[PVR_ST_C_P] = clampd(c0, 1e-3, 1.0 - 1e-3);
    }
}

// 5 + 6: M-step sums of the participating patches, potentials, eligibility.
// bpart = {sum p, sum p e^2, sum pbar, sum pbar^2, n_elig, min pbar, max pbar}
__global__ void __launch_bounds__(256) k_em_patch_pot(const int32_t *__restrict__ desc, int n, int tpp,
                                                      const uint8_t *__restrict__ mask_in,
                                                      const double *__restrict__ part,
                                                      double min_valid_frac, double *__restrict__ pbar,
                                                      uint8_t *__restrict__ elig,
                                                      double *__restrict__ bpart, double *__restrict__ state,
                                                      double *__restrict__ pstat, double c0, int rule,
                                                      unsigned *__restrict__ counter)
{
    __shared__ double sh[32 * 5];
    double a[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, mn[1] = {INFINITY}, mx[1] = {-INFINITY};
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        double sp = 0.0, spe2 = 0.0, sp2 = 0.0, nv = 0.0;
        for (int t = 0; t < tpp; ++t) {
            const double *pt = part + ((size_t)p * tpp + t) * kPartStride;
            sp += pt[4];
            spe2 += pt[5];
            sp2 += pt[6];
            nv += pt[7];
        }
        if (!mask_in || mask_in[p]) {
            a[0] += sp;
            a[1] += spe2;
        }
        const int32_t *d = desc + 8 * (size_t)p;
        double npx = (double)d[4] * (double)d[5];
        double pb = nv > 0.0 ? sqrt(sp2 / nv) : 0.0;
        bool el = nv > 0.0 && nv >= min_valid_frac * npx;
        pbar[p] = pb;
        elig[p] = el ? 1 : 0;
        if (el) {
            a[2] += pb;
            a[3] += pb * pb;
            a[4] += 1.0;
            mn[0] = fmin(mn[0], pb);
            mx[0] = fmax(mx[0], pb);
        }
    }
    block_reduce<5>(a, sh, 0);
    block_reduce<1>(mn, sh, 1);
    block_reduce<1>(mx, sh, 2);
    double v[7] = {a[0], a[1], a[2], a[3], a[4], mn[0], mx[0]};
    store_block(bpart, v, 7);
    if (last_block(counter) && threadIdx.x < 32) em_patch_head(gridDim.x, bpart, state, pstat, c0, rule);
}

// M-step of the patch-level model (called by the 32 lanes of warp 0 of the
// last block); stops the loop when m_p = 0 or no weight.
__device__ void em_patch_mstep(int nb, const double *__restrict__ bpart, double *__restrict__ state,
                               double *__restrict__ pstat)
{
    const bool lead = (threadIdx.x & 31) == 0;
    const double stop = pstat[6], mp = pstat[5];
    __syncwarp();   // every lane has read the flags before lane 0 may write them
    if (stop != 0.0) return;
    if (mp == 0.0) {
        if (lead) pstat[6] = 1.0;
        return;
    }
    const double sw = warp_fold(nb, bpart, 0, 0), swp = warp_fold(nb, bpart, 1, 0);
    const double swp2 = warp_fold(nb, bpart, 2, 0);
    if (!lead) return;
    if (!(sw > 0.0)) {
        pstat[6] = 1.0;
        return;
    }
    double mu = swp / sw;
    double v2 = swp2 / sw - mu * mu;
    state[PVR_ST_MU_P] = mu;
    state[PVR_ST_SIGMA2_P] = v2 < 1e-4 ? 1e-4 : v2;
    state[PVR_ST_C_P] = clampd(sw / pstat[7], 1e-3, 1.0 - 1e-3);
}

// E-step of the patch-level model: w = G c_p / (G c_p + m_p (1 - c_p)),
// G the one-sided Gaussian density of pbar; w = 1 if m_p = 0; 0 if not
// eligible.  bpart = {sum w, sum w pbar, sum w pbar^2} over eligible patches.
__device__ void em_patch_estep_block(int n, const uint8_t *__restrict__ elig, const double *__restrict__ pbar,
                                     const double *__restrict__ state, const double *__restrict__ pstat,
                                     double *__restrict__ wsc, double *__restrict__ bpart, double *sh)
{
    const double mu = state[PVR_ST_MU_P], v2 = state[PVR_ST_SIGMA2_P], cp = state[PVR_ST_C_P];
    const double mp = pstat[5];
    const double gnorm = 1.0 / (sqrt(2.0 * 3.14159265358979323846) * sqrt(v2));
    double a[3] = {0.0, 0.0, 0.0};
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        double wv;
        if (!elig[p]) {
            wv = 0.0;
        } else if (mp == 0.0) {
            wv = 1.0;
        } else {
            double dl = pbar[p] >= mu ? 0.0 : pbar[p] - mu;
            double G = exp(-(dl * dl) / (2.0 * v2)) * gnorm;
            wv = (G * cp) / (G * cp + mp * (1.0 - cp));
        }
        wsc[p] = wv;
        if (elig[p]) {
            a[0] += wv;
            a[1] += wv * pbar[p];
            a[2] += wv * pbar[p] * pbar[p];
        }
    }
    block_reduce<3>(a, sh, 0);
    store_block(bpart, a, 3);
}

// With mstep, the last block to finish runs the M-step on the partials.
__global__ void __launch_bounds__(256) k_em_patch_estep(int n, const uint8_t *__restrict__ elig,
                                                        const double *__restrict__ pbar,
                                                        double *__restrict__ state,
                                                        double *__restrict__ pstat,
                                                        double *__restrict__ wsc,
                                                        double *__restrict__ bpart, int mstep,
                                                        unsigned *__restrict__ counter)
{
    __shared__ double sh[32 * 3];
    // the loop has stopped: keep the last weights (every block still counts in)
    if (pstat[6] == 0.0) em_patch_estep_block(n, elig, pbar, state, pstat, wsc, bpart, sh);
    if (last_block(counter) && mstep && threadIdx.x < 32) em_patch_mstep(gridDim.x, bpart, state, pstat);
}

// Fold of k_em_patch_final (the 32 lanes of warp 0 of the last block):
// patch counts into the EM state.
__device__ void em_patch_tail(int nb, const double *__restrict__ bpart, double *__restrict__ state,
                              const double *__restrict__ pstat, int rule)
{
    const double nin = warp_fold(nb, bpart, 0, 0);
    if ((threadIdx.x & 31) != 0) return;
    state[PVR_ST_N_ELIG] = pstat[7];
    state[PVR_ST_N_IN] = nin;
    if (rule == 0) state[PVR_ST_M_P] = pstat[5];
    state[PVR_ST_INIT] = 1.0;
}

// Masks and outputs; bpart[0] = number of inlier patches of the block.
__global__ void __launch_bounds__(256) k_em_patch_final(int n, const uint8_t *__restrict__ elig,
                                                        const double *__restrict__ pbar,
                                                        const double *__restrict__ wsc, int rule,
                                                        double threshold,
                                                        uint8_t *__restrict__ mask_out,
                                                        float *__restrict__ w_patch,
                                                        float *__restrict__ pbar_out,
                                                        double *__restrict__ bpart, double *__restrict__ state,
                                                        const double *__restrict__ pstat,
                                                        unsigned *__restrict__ counter)
{
    __shared__ double sh[32];
    double cnt[1] = {0.0};
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        double wv = rule == 1 ? (elig[p] ? pbar[p] : 0.0) : wsc[p];
        uint8_t m = rule == 1 ? (elig[p] && pbar[p] >= threshold) : (elig[p] && wsc[p] >= 0.5);
        mask_out[p] = m;
        cnt[0] += m;
        if (w_patch) w_patch[p] = (float)wv;
        if (pbar_out) pbar_out[p] = (float)pbar[p];
    }
    block_reduce<1>(cnt, sh, 0);
    store_block(bpart, cnt, 1);
    if (last_block(counter) && threadIdx.x < 32) em_patch_tail(gridDim.x, bpart, state, pstat, rule);
}


// Weighted SIRT step (rows of A sum to one): x <- max(x + alpha addon / conf, 0)
// where conf > eps; init_mode: x <- conf > eps ? addon / conf : 0.  Optionally
// zeroes the accumulators for the next pass.  Vectorised by 4.
__global__ void __launch_bounds__(256) k_volume_update(float *__restrict__ x,
                                                       float *__restrict__ addon,
                                                       float *__restrict__ conf, long long n,
                                                       float alpha, float eps, int clear,
                                                       int init_mode)
{
    long long n4 = n >> 2;
    long long stride = (long long)gridDim.x * blockDim.x;
    float4 *x4 = reinterpret_cast<float4 *>(x);
    float4 *a4 = reinterpret_cast<float4 *>(addon);
    float4 *c4 = reinterpret_cast<float4 *>(conf);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 a = a4[i], c = c4[i], v = init_mode ? z4 : x4[i];
        float *vp = &v.x;
        const float *ap = &a.x, *cp = &c.x;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (cp[k] > eps) {
                if (init_mode) vp[k] = ap[k] / cp[k];
                else vp[k] = fmaxf(vp[k] + alpha * ap[k] / cp[k], 0.f);
            }
        }
        x4[i] = v;
        if (clear) {
            a4[i] = z4;
            c4[i] = z4;
        }
    }
    for (long long i = (n4 << 2) + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        float a = addon[i], c = conf[i];
        float v = init_mode ? 0.f : x[i];
        if (c > eps) v = init_mode ? a / c : fmaxf(v + alpha * a / c, 0.f);
        x[i] = v;
        if (clear) addon[i] = conf[i] = 0.f;
    }
}

// The same step on interleaved (addon, conf) pairs (the adjoint's own
// accumulator layout: one vector reduction per voxel and sample corner).
__global__ void __launch_bounds__(256) k_volume_update_pairs(float *__restrict__ x,
                                                             float2 *__restrict__ acc, long long n,
                                                             float alpha, float eps, int clear,
                                                             int init_mode)
{
    long long stride = (long long)gridDim.x * blockDim.x;
    long long n2 = n >> 1;
    float2 *x2 = reinterpret_cast<float2 *>(x);
    float4 *a4 = reinterpret_cast<float4 *>(acc);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += stride) {
        float4 a = a4[i];   // (addon, conf) of voxels 2i and 2i+1
        float2 v = init_mode ? make_float2(0.f, 0.f) : x2[i];
        if (a.y > eps) v.x = init_mode ? a.x / a.y : fmaxf(v.x + alpha * a.x / a.y, 0.f);
        if (a.w > eps) v.y = init_mode ? a.z / a.w : fmaxf(v.y + alpha * a.z / a.w, 0.f);
        x2[i] = v;
        if (clear) a4[i] = z4;
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        long long i = n - 1;
        float2 a = acc[i];
        float v = init_mode ? 0.f : x[i];
        if (a.y > eps) v = init_mode ? a.x / a.y : fmaxf(v + alpha * a.x / a.y, 0.f);
        x[i] = v;
        if (clear) acc[i] = make_float2(0.f, 0.f);
    }
}

__global__ void __launch_bounds__(256) k_split_pairs(const float2 *__restrict__ acc, long long n,
                                                     float *__restrict__ addon,
                                                     float *__restrict__ conf, int accumulate)
{
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        float2 a = acc[i];
        if (addon) addon[i] = accumulate ? addon[i] + a.x : a.x;
        if (conf) conf[i] = accumulate ? conf[i] + a.y : a.y;
    }
}

// ---------------------------------------------------------- registration --

__global__ void k_reg_init(const double *__restrict__ poses, int n_params, int n, double *__restrict__ best,
                           double *__restrict__ trial, double *__restrict__ delta,
                           int32_t *__restrict__ active, double delta0)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    for (int k = 0; k < n_params; ++k) {
        double v = poses[(size_t)n_params * p + k];
        best[kRegStride * (size_t)p + k] = v;
        trial[(size_t)n_params * p + k] = v;
    }
    delta[p] = delta0;
    active[p] = 1;
}

// Assess evaluation `eval` (NCC and gradient at the trial pose) and propose
// the next trial: best + delta (g/s) / |g/s| / s, s = per-parameter scale
// (translations 1 mm; rigid angles the patch half-diagonal times pi/180,
// affine entries the half-diagonal, so that one scaled unit moves the patch
// edge by about 1 mm).
__global__ void k_reg_step(const DevGeom *__restrict__ g, const int32_t *__restrict__ desc, int n_params,
                           int n, int eval, int last, const double *__restrict__ ncc,
                           const double *__restrict__ grad, double *__restrict__ best,
                           double *__restrict__ gbest, double *__restrict__ nbest,
                           double *__restrict__ trial, double *__restrict__ delta,
                           int32_t *__restrict__ active, double delta_min, double grow, int fixed)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || !active[p]) return;
    double *b = best + kRegStride * (size_t)p;
    double *gb = gbest + kRegStride * (size_t)p;
    double *tr = trial + (size_t)n_params * p;
    // grad is null on the last evaluation (no further step uses it)
    const double *gr = grad ? grad + (size_t)n_params * p : nullptr;
    double v = ncc[p];
    if (eval == 0) {
        nbest[p] = v;
        if (gr)
            for (int k = 0; k < n_params; ++k) gb[k] = gr[k];
        if (v == 0.0) {
            active[p] = 0;
            return;
        }
    } else if (fixed || v > nbest[p]) {
        for (int k = 0; k < n_params; ++k) {
            b[k] = tr[k];
            if (gr) gb[k] = gr[k];
        }
        nbest[p] = v;
        if (!fixed) delta[p] = __dmul_rn(delta[p], grow);
    } else {
        delta[p] = __dmul_rn(delta[p], 0.5);
        if (delta[p] < delta_min) {
            active[p] = 0;
            return;
        }
    }
    if (last) return;
    const int32_t *d = desc + 8 * (size_t)p;
    const double *S = g->p2w[d[0]];
    double cw = sqrt(S[0] * S[0] + S[4] * S[4] + S[8] * S[8]) * (double)d[4];
    double ch = sqrt(S[1] * S[1] + S[5] * S[5] + S[9] * S[9]) * (double)d[5];
    double hd = 0.5 * sqrt(cw * cw + ch * ch);
    const double sl = n_params == 12 ? hd : hd * (3.14159265358979323846 / 180.0);
    double gn = 0.0;
    for (int k = 0; k < n_params; ++k) {
        const double sk = k < 3 ? 1.0 : sl;
        gn = __dadd_rn(gn, __dmul_rn(__ddiv_rn(gb[k], sk), __ddiv_rn(gb[k], sk)));
    }
    gn = __dsqrt_rn(gn);
    if (!(gn > 0.0)) {
        active[p] = 0;
        return;
    }
    for (int k = 0; k < n_params; ++k) {
        const double sk = k < 3 ? 1.0 : sl;
        tr[k] = __dadd_rn(b[k], __ddiv_rn(__ddiv_rn(__dmul_rn(delta[p], __ddiv_rn(gb[k], sk)), gn), sk));
    }
}

__global__ void k_reg_finish(const double *__restrict__ best, const double *__restrict__ nbest,
                             int n_params, int n, double *__restrict__ poses, double *__restrict__ ncc_out)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    for (int k = 0; k < n_params; ++k) poses[(size_t)n_params * p + k] = best[kRegStride * (size_t)p + k];
    if (ncc_out) ncc_out[p] = nbest[p];
}

}  // namespace

cudaError_t launch_em_stats(const float *y, const float *sim, const uint8_t *valid,
                            const int32_t *desc, int n, int64_t n_pix, const Tiling &tl,
                            int32_t *err, double *part, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_em_stats<<<(unsigned)n * tl.tpp, 256, 0, st>>>(y, sim, valid, desc, tl, (long long)n_pix,
                                                     err, part);
    return cudaGetLastError();
}

cudaError_t launch_em(const float *y, const float *sim, const uint8_t *valid, const int32_t *desc,
                      int n, int64_t n_pix, const Tiling &tl, int32_t *err, double *state,
                      const uint8_t *mask_in, uint8_t *mask_out, float *p, float *w_patch,
                      float *pbar_out, double *part, double *pstat, double *pbar, double *wsc,
                      uint8_t *elig, double *bpart, unsigned *counter, const pvr_params &prm, cudaStream_t st)
{
    k_em_prepare<<<1, kRedThreads, 0, st>>>(n, tl.tpp, mask_in, part, state, pstat, prm.em_c0,
                                            prm.em_sigma_floor_rel);
    if (n > 0)
        k_em_estep<<<(unsigned)n * tl.tpp, 256, 0, st>>>(y, sim, valid, desc, tl, (long long)n_pix,
                                                         err, mask_in, pstat, p, part);
    int nb = (n + 255) / 256;
    if (nb > kEmBlockMax) nb = kEmBlockMax;
    if (nb < 1) nb = 1;
    const int rule = prm.patch_rule == 1 ? 1 : 0;
    // each patch-level kernel's last block runs the fold that follows it
    // (head, M-step, tail) on the block partials; the arrival counter returns
    // to 0 after every such kernel, and is zeroed here as well so that a call
    // after an aborted one starts clean
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    k_em_patch_pot<<<nb, 256, 0, st>>>(desc, n, tl.tpp, mask_in, part, prm.em_min_valid_frac, pbar,
                                       elig, bpart, state, pstat, prm.em_c0, rule, counter);
    if (rule == 0) {
        for (int it = 0; it <= prm.patch_em_iters; ++it)
            k_em_patch_estep<<<nb, 256, 0, st>>>(n, elig, pbar, state, pstat, wsc, bpart,
                                                 it < prm.patch_em_iters, counter);
    }
    k_em_patch_final<<<nb, 256, 0, st>>>(n, elig, pbar, wsc, rule, prm.patch_threshold, mask_out,
                                         w_patch, pbar_out, bpart, state, pstat, counter);
    return cudaGetLastError();
}

// Number of kernel launches launch_em makes.
int em_launch_count(int n, const pvr_params &prm)
{
    return (n > 0 ? 2 : 1) + 1 + (prm.patch_rule == 1 ? 0 : prm.patch_em_iters + 1) + 1;
}

cudaError_t launch_volume_update(float *x, float *addon, float *conf, int64_t nvox, float alpha,
                                 float conf_eps, int clear, int init_mode, cudaStream_t st)
{
    if (nvox <= 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long n4 = (nvox + 3) / 4;
    long long blocks = (n4 + 255) / 256;
    long long cap = (long long)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_volume_update<<<(unsigned)blocks, 256, 0, st>>>(x, addon, conf, (long long)nvox, alpha,
                                                      conf_eps, clear, init_mode);
    return cudaGetLastError();
}

static unsigned elementwise_blocks(long long work)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (work + 255) / 256, cap = (long long)sms * 8;
    if (blocks > cap) blocks = cap;
    return (unsigned)(blocks < 1 ? 1 : blocks);
}

cudaError_t launch_volume_update_pairs(float *x, float2 *acc, int64_t nvox, float alpha,
                                       float conf_eps, int clear, int init_mode, cudaStream_t st)
{
    if (nvox <= 0) return cudaSuccess;
    k_volume_update_pairs<<<elementwise_blocks(nvox / 2 + 1), 256, 0, st>>>(
        x, acc, (long long)nvox, alpha, conf_eps, clear, init_mode);
    return cudaGetLastError();
}

cudaError_t launch_split_pairs(const float2 *acc, int64_t nvox, float *addon, float *conf,
                               int accumulate, cudaStream_t st)
{
    if (nvox <= 0) return cudaSuccess;
    k_split_pairs<<<elementwise_blocks(nvox), 256, 0, st>>>(acc, (long long)nvox, addon, conf,
                                                            accumulate);
    return cudaGetLastError();
}

cudaError_t launch_reg_init(const double *poses, int n_params, int n, double *best, double *trial, double *delta,
                            int32_t *active, double delta0, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_reg_init<<<(n + 127) / 128, 128, 0, st>>>(poses, n_params, n, best, trial, delta, active, delta0);
    return cudaGetLastError();
}

cudaError_t launch_reg_step(const DevGeom *g, const int32_t *desc, int n, int eval, int last,
                            const double *ncc, const double *grad, double *best, double *gbest,
                            double *nbest, double *trial, double *delta, int32_t *active,
                            const pvr_params &prm, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_reg_step<<<(n + 127) / 128, 128, 0, st>>>(g, desc, prm.n_params, n, eval, last, ncc, grad, best, gbest,
                                                nbest, trial, delta, active, prm.reg_delta_min,
                                                prm.reg_grow, prm.reg_fixed_step);
    return cudaGetLastError();
}

cudaError_t launch_reg_finish(const double *best, const double *nbest, int n_params, int n, double *poses,
                              double *ncc_out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_reg_finish<<<(n + 127) / 128, 128, 0, st>>>(best, nbest, n_params, n, poses, ncc_out);
    return cudaGetLastError();
}

}  // namespace pvr
