// Kernels of the learned pose proposal: a small 2-D CNN over (acquired
// patch, simulated patch) pairs that predicts the rigid correction of the
// patch pose.  Activations and weights are bfloat16 (NHWC, channels a
// multiple of 16), accumulation float32.
//
// Every 3x3 convolution pass is one implicit GEMM on the tensor cores
// (mma.sync m16n8k16, bf16 x bf16 -> f32), with the im2col gather folded
// into the tile loads:
//   forward      C[m = (n, oy, ox)][co]       = sum_k A[m][k = (ky, kx, ci)] B[co][k]
//   input grad   C[m = (n, iy, ix)][ci]       = sum_k A[m][k = (ky, kx, co)] B[ci][k]
//   weight grad  C[co][(ky, kx, ci)]          = sum_{m = (n, oy, ox)} A[co][m] B[(ky, kx, ci)][m]
// The tile loader of each pass turns (row, k0) into 8 consecutive k values.
#include <cuda_bf16.h>

#include "pvr_internal.h"

namespace pvr {
namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16;
constexpr int kRowStride = 24;   // bf16 per shared-memory tile row (16 used): conflict-free fragment reads

struct ConvShape {
    int B, IH, IW, Cin, OH, OW, Cout, stride;   // padding 1, 3x3 taps
};

__device__ __forceinline__ uint4 zero4() { return make_uint4(0u, 0u, 0u, 0u); }

__device__ __forceinline__ unsigned pack2(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

// ---- tile loaders: 8 consecutive k of one row (uint4 = 8 bf16) ----

// forward A: activations at (n, oy*s+ky-1, ox*s+kx-1, ci..ci+7); k = (ky*3+kx)*Cin + ci
struct FwdA {
    const __nv_bfloat16 *in;
    ConvShape sh;
    __device__ uint4 operator()(long long m, int k0, long long M, int K) const
    {
        if (m >= M || k0 >= K) return zero4();
        const int tap = k0 / sh.Cin, ci = k0 - tap * sh.Cin, ky = tap / 3, kx = tap - ky * 3;
        const int ox = (int)(m % sh.OW);
        const long long r = m / sh.OW;
        const int oy = (int)(r % sh.OH), n = (int)(r / sh.OH);
        const int iy = oy * sh.stride + ky - 1, ix = ox * sh.stride + kx - 1;
        if (iy < 0 || ix < 0 || iy >= sh.IH || ix >= sh.IW) return zero4();
        return *reinterpret_cast<const uint4 *>(in + (((size_t)n * sh.IH + iy) * sh.IW + ix) * sh.Cin + ci);
    }
};

// forward B: weights w[co][ky][kx][ci], row co, 8 consecutive k
struct FwdB {
    const __nv_bfloat16 *w;
    __device__ uint4 operator()(long long co, int k0, long long N, int K) const
    {
        if (co >= N || k0 >= K) return zero4();
        return *reinterpret_cast<const uint4 *>(w + (size_t)co * K + k0);
    }
};

// input-grad A: upstream gradient g(n, oy, ox, co) times the ReLU mask of
// the layer output, at the output position that tap (ky, kx) of input
// (iy, ix) feeds; k = (ky*3+kx)*Cout + co
struct BwdA {
    const __nv_bfloat16 *g, *out;
    ConvShape sh;
    __device__ uint4 operator()(long long m, int k0, long long M, int K) const
    {
        if (m >= M || k0 >= K) return zero4();
        const int tap = k0 / sh.Cout, co = k0 - tap * sh.Cout, ky = tap / 3, kx = tap - ky * 3;
        const int ix = (int)(m % sh.IW);
        const long long r = m / sh.IW;
        const int iy = (int)(r % sh.IH), n = (int)(r / sh.IH);
        const int ty = iy + 1 - ky, tx = ix + 1 - kx;
        if (ty < 0 || tx < 0 || ty % sh.stride || tx % sh.stride) return zero4();
        const int oy = ty / sh.stride, ox = tx / sh.stride;
        if (oy >= sh.OH || ox >= sh.OW) return zero4();
        const size_t o = (((size_t)n * sh.OH + oy) * sh.OW + ox) * sh.Cout + co;
        uint4 gv = *reinterpret_cast<const uint4 *>(g + o), ov = *reinterpret_cast<const uint4 *>(out + o);
        const __nv_bfloat16 *gp = reinterpret_cast<const __nv_bfloat16 *>(&gv);
        const __nv_bfloat16 *op = reinterpret_cast<const __nv_bfloat16 *>(&ov);
        unsigned u[4];
        const __nv_bfloat16 zero = __float2bfloat16(0.f);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            __nv_bfloat16 a = __bfloat162float(op[2 * j]) > 0.f ? gp[2 * j] : zero;
            __nv_bfloat16 b = __bfloat162float(op[2 * j + 1]) > 0.f ? gp[2 * j + 1] : zero;
            u[j] = pack2(a, b);
        }
        return make_uint4(u[0], u[1], u[2], u[3]);
    }
};

// input-grad B: w[co][ky][kx][ci] as B[ci][k = (ky, kx, co)]: 8 consecutive co
struct BwdB {
    const __nv_bfloat16 *w;
    ConvShape sh;
    __device__ uint4 operator()(long long ci, int k0, long long N, int K) const
    {
        if (ci >= N || k0 >= K) return zero4();
        const int tap = k0 / sh.Cout, co = k0 - tap * sh.Cout;
        const size_t K9 = 9 * (size_t)sh.Cin;
        unsigned u[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            u[j] = pack2(w[(size_t)(co + 2 * j) * K9 + (size_t)tap * sh.Cin + ci],
                         w[(size_t)(co + 2 * j + 1) * K9 + (size_t)tap * sh.Cin + ci]);
        return make_uint4(u[0], u[1], u[2], u[3]);
    }
};

// weight-grad A: masked upstream gradient as A[co][m]: 8 consecutive m
struct WgA {
    const __nv_bfloat16 *g, *out;
    int Cout;
    __device__ uint4 operator()(long long co, int m0, long long N, int K) const
    {
        unsigned u[4];
        const __nv_bfloat16 zero = __float2bfloat16(0.f);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            __nv_bfloat16 v[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = m0 + 2 * j + h;
                v[h] = zero;
                if (co < N && m < K) {
                    const size_t o = (size_t)m * Cout + co;
                    if (__bfloat162float(out[o]) > 0.f) v[h] = g[o];
                }
            }
            u[j] = pack2(v[0], v[1]);
        }
        return make_uint4(u[0], u[1], u[2], u[3]);
    }
};

// weight-grad B: activations as B[k9 = (ky, kx, ci)][m]: 8 consecutive m
struct WgB {
    const __nv_bfloat16 *in;
    ConvShape sh;
    __device__ uint4 operator()(long long k9, int m0, long long N, int K) const
    {
        unsigned u[4];
        const __nv_bfloat16 zero = __float2bfloat16(0.f);
        const int tap = (int)(k9 / sh.Cin), ci = (int)(k9 - (long long)tap * sh.Cin);
        const int ky = tap / 3, kx = tap - ky * 3;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            __nv_bfloat16 v[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = m0 + 2 * j + h;
                v[h] = zero;
                if (k9 < N && m < K) {
                    const int ox = m % sh.OW, r = m / sh.OW, oy = r % sh.OH, n = r / sh.OH;
                    const int iy = oy * sh.stride + ky - 1, ix = ox * sh.stride + kx - 1;
                    if (iy >= 0 && ix >= 0 && iy < sh.IH && ix < sh.IW)
                        v[h] = in[(((size_t)n * sh.IH + iy) * sh.IW + ix) * sh.Cin + ci];
                }
            }
            u[j] = pack2(v[0], v[1]);
        }
        return make_uint4(u[0], u[1], u[2], u[3]);
    }
};

// ---- epilogues: the 4 accumulator values of a fragment ----

// bias + ReLU, bf16 NHWC store
struct EpAct {
    __nv_bfloat16 *out;
    const float *bias;
    int N;
    __device__ void operator()(long long m, long long n, float v) const
    {
        out[(size_t)m * N + n] = __float2bfloat16(fmaxf(v + bias[n], 0.f));
    }
};

// plain bf16 store (input gradient)
struct EpStore {
    __nv_bfloat16 *out;
    int N;
    __device__ void operator()(long long m, long long n, float v) const
    {
        out[(size_t)m * N + n] = __float2bfloat16(v);
    }
};

// float32 accumulation of split-K partial sums (weight gradient)
struct EpAdd {
    float *out;
    int N;
    __device__ void operator()(long long m, long long n, float v) const
    {
        atomicAdd(out + (size_t)m * N + n, v);
    }
};

__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C[M][N] (+)= A[M][K] B[N][K]^T over the K range of this CTA (blockIdx.z
// selects a slice of k_per_split); 128 threads, 64x64 tile, warp w owns
// rows 16w..16w+15 and all 64 columns (8 m16n8 fragments).
template <class LA, class LB, class EP>
__global__ void __launch_bounds__(128) k_gemm_bf16(LA la, LB lb, EP ep, long long M, long long N, int K,
                                                   int k_per_split)
{
    __shared__ __align__(16) __nv_bfloat16 As[kBM * kRowStride];
    __shared__ __align__(16) __nv_bfloat16 Bs[kBN * kRowStride];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const long long m0 = (long long)blockIdx.x * kBM, n0 = (long long)blockIdx.y * kBN;
    const int kb = blockIdx.z * k_per_split;
    const int ke = min(K, kb + k_per_split);
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    // each thread loads one 8-value chunk of each tile: row tid / 2, half tid % 2
    const int lr = tid >> 1, lh = (tid & 1) * 8;
    for (int k = kb; k < ke; k += kBK) {
        const uint4 av = la(m0 + lr, k + lh, M, ke);
        const uint4 bv = lb(n0 + lr, k + lh, N, ke);
        __syncthreads();
        *reinterpret_cast<uint4 *>(As + lr * kRowStride + lh) = av;
        *reinterpret_cast<uint4 *>(Bs + lr * kRowStride + lh) = bv;
        __syncthreads();
        const __nv_bfloat16 *ar = As + (warp * 16 + g) * kRowStride;
        unsigned a[4];
        a[0] = *reinterpret_cast<const unsigned *>(ar + 2 * t);
        a[1] = *reinterpret_cast<const unsigned *>(ar + 8 * kRowStride + 2 * t);
        a[2] = *reinterpret_cast<const unsigned *>(ar + 2 * t + 8);
        a[3] = *reinterpret_cast<const unsigned *>(ar + 8 * kRowStride + 2 * t + 8);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const __nv_bfloat16 *br = Bs + (j * 8 + g) * kRowStride;
            const unsigned b0 = *reinterpret_cast<const unsigned *>(br + 2 * t);
            const unsigned b1 = *reinterpret_cast<const unsigned *>(br + 2 * t + 8);
            mma_bf16(acc[j], a, b0, b1);
        }
    }
    const long long r0 = m0 + warp * 16 + g;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const long long c0 = n0 + j * 8 + 2 * t;
        if (r0 < M) {
            if (c0 < N) ep(r0, c0, acc[j][0]);
            if (c0 + 1 < N) ep(r0, c0 + 1, acc[j][1]);
        }
        if (r0 + 8 < M) {
            if (c0 < N) ep(r0 + 8, c0, acc[j][2]);
            if (c0 + 1 < N) ep(r0 + 8, c0 + 1, acc[j][3]);
        }
    }
}

// Network input: per patch, the acquired and simulated 64x64 patches, each
// normalised to zero mean and unit deviation over the valid pixels
// (invalid pixels 0), as channels 0 and 1 of a 16-channel bf16 NHWC image.
__global__ void __launch_bounds__(256) k_cnn_input(const float *__restrict__ y, const float *__restrict__ s,
                                                   const uint8_t *__restrict__ valid,
                                                   const int32_t *__restrict__ desc, int first, long long n_pix,
                                                   __nv_bfloat16 *__restrict__ img)
{
    __shared__ float red[32 * 5];
    const int b = blockIdx.x;
    const int32_t *d = desc + 8 * (size_t)(first + b);
    const size_t off = (size_t)d[6];
    const int n = 64 * 64;
    // only 64x64 patches inside the pixel arrays are read; others stay empty
    const bool fits = d[4] == 64 && d[5] == 64 && d[6] >= 0 && (long long)off + n <= n_pix;
    float v[5] = {0, 0, 0, 0, 0};
    for (int t = threadIdx.x; fits && t < n; t += blockDim.x) {
        if (!valid[off + t]) continue;
        const float a = y[off + t], c = s[off + t];
        v[0] += 1.f;
        v[1] += a;
        v[2] += a * a;
        v[3] += c;
        v[4] += c * c;
    }
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 5; ++k) red[(threadIdx.x >> 5) * 5 + k] = v[k];
    __syncthreads();
    float tot[5] = {0, 0, 0, 0, 0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
        for (int k = 0; k < 5; ++k) tot[k] += red[w * 5 + k];
    const float cnt = fmaxf(tot[0], 1.f);
    const float my = tot[1] / cnt, ms = tot[3] / cnt;
    const float sy = rsqrtf(fmaxf(tot[2] / cnt - my * my, 1e-6f)), ss = rsqrtf(fmaxf(tot[4] / cnt - ms * ms, 1e-6f));
    __nv_bfloat16 *o = img + (size_t)b * n * 16;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const bool ok = fits && valid[off + t];
        __nv_bfloat16 px[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) px[c] = zero;
        if (ok) {
            px[0] = __float2bfloat16((y[off + t] - my) * sy);
            px[1] = __float2bfloat16((s[off + t] - ms) * ss);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(o + (size_t)t * 16);
        dst[0] = *reinterpret_cast<const uint4 *>(px);
        dst[1] = *reinterpret_cast<const uint4 *>(px + 8);
    }
}

// Head: global mean of the last activation (B x P x C, P positions), then
// out[b][j] = bias[j] + sum_c wl[j][c] mean[b][c] (float32).  One CTA per
// sample, C <= 128 threads.
__global__ void k_head_forward(const __nv_bfloat16 *__restrict__ act, int P, int C,
                               const float *__restrict__ wl, const float *__restrict__ bl, int J,
                               float *__restrict__ pooled, float *__restrict__ out)
{
    __shared__ float m[128];
    const int b = blockIdx.x, c = threadIdx.x;
    if (c < C) {
        float s = 0.f;
        for (int p = 0; p < P; ++p) s += __bfloat162float(act[((size_t)b * P + p) * C + c]);
        m[c] = s / P;
        pooled[(size_t)b * C + c] = m[c];
    }
    __syncthreads();
    if (c < J) {
        float s = bl[c];
        for (int k = 0; k < C; ++k) s = fmaf(wl[c * C + k], m[k], s);
        out[(size_t)b * J + c] = s;
    }
}

// Head backward for the loss mean_b sum_j (out - target)^2 / B: gradients
// of the linear layer (accumulated into gwl, gbl) and of the last
// activation (bf16, spread evenly over the P positions).
__global__ void k_head_backward(const float *__restrict__ out, const float *__restrict__ target, int B,
                                int J, const float *__restrict__ pooled, const float *__restrict__ wl,
                                int C, int P, float *__restrict__ gwl, float *__restrict__ gbl,
                                __nv_bfloat16 *__restrict__ gact, float *__restrict__ loss)
{
    __shared__ float go[16];
    const int b = blockIdx.x, c = threadIdx.x;
    if (c < J) {
        const float e = out[(size_t)b * J + c] - target[(size_t)b * J + c];
        go[c] = 2.f * e / B;
        atomicAdd(loss, e * e / B);
        atomicAdd(gbl + c, go[c]);
    }
    __syncthreads();
    if (c < C) {
        float gm = 0.f;
        for (int j = 0; j < J; ++j) {
            gm = fmaf(wl[j * C + c], go[j], gm);
            atomicAdd(gwl + j * C + c, go[j] * pooled[(size_t)b * C + c]);
        }
        const __nv_bfloat16 gv = __float2bfloat16(gm / P);
        for (int p = 0; p < P; ++p) gact[((size_t)b * P + p) * C + c] = gv;
    }
}

// Bias gradient of a convolution: sum over m of the masked upstream gradient.
__global__ void k_bias_grad(const __nv_bfloat16 *__restrict__ g, const __nv_bfloat16 *__restrict__ out,
                            long long M, int C, float *__restrict__ gb)
{
    const int c = blockIdx.y;
    float s = 0.f;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < M; m += (long long)gridDim.x * blockDim.x) {
        const size_t o = (size_t)m * C + c;
        if (__bfloat162float(out[o]) > 0.f) s += __bfloat162float(g[o]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(gb + c, s);
}

// Adam step on float32 master weights; refreshes the bf16 copy (may be null).
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ gw, float *__restrict__ m1,
                       float *__restrict__ m2, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2, __nv_bfloat16 *__restrict__ wb)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gr = gw[i];
        const float a = fmaf(b1, m1[i], (1.f - b1) * gr), b = fmaf(b2, m2[i], (1.f - b2) * gr * gr);
        m1[i] = a;
        m2[i] = b;
        const float v = w[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
        w[i] = v;
        if (wb) wb[i] = __float2bfloat16(v);
    }
}

__global__ void k_to_bf16(const float *__restrict__ a, __nv_bfloat16 *__restrict__ b, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16(a[i]);
}

// trial[p][k] = poses[p][k] + scale[k] * out[p][k] (network correction in
// pose units)
__global__ void k_propose_trial(const double *__restrict__ poses, const float *__restrict__ out, int n,
                                double s0, double s1, double s2, double s3, double s4, double s5,
                                double *__restrict__ trial)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6 * n) return;
    const int k = i % 6;
    const double sc = k == 0 ? s0 : k == 1 ? s1 : k == 2 ? s2 : k == 3 ? s3 : k == 4 ? s4 : s5;
    trial[i] = poses[i] + sc * (double)out[i];
}

// Keep the proposal where it raises NCC, else the plain pose.
__global__ void k_propose_select(const double *__restrict__ ncc0, const double *__restrict__ ncc1,
                                 const double *__restrict__ trial, int n, double *__restrict__ poses,
                                 int32_t *__restrict__ accepted)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const bool take = ncc1[p] > ncc0[p];
    if (take)
        for (int k = 0; k < 6; ++k) poses[6 * (size_t)p + k] = trial[6 * (size_t)p + k];
    if (accepted) accepted[p] = take ? 1 : 0;
}

template <class LA, class LB, class EP>
cudaError_t gemm(LA la, LB lb, EP ep, long long M, long long N, int K, int split, cudaStream_t st)
{
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    int kps = (K + split - 1) / split;
    kps = (kps + kBK - 1) / kBK * kBK;
    const int nz = (K + kps - 1) / kps;
    dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + kBN - 1) / kBN), (unsigned)nz);
    k_gemm_bf16<LA, LB, EP><<<grid, 128, 0, st>>>(la, lb, ep, M, N, K, kps);
    return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------------------- launchers --

cudaError_t cnn_conv_forward(const __nv_bfloat16 *in, const __nv_bfloat16 *w, const float *bias,
                             __nv_bfloat16 *out, int B, int IH, int IW, int Cin, int Cout, int stride,
                             cudaStream_t st)
{
    ConvShape sh{B, IH, IW, Cin, (IH - 1) / stride + 1, (IW - 1) / stride + 1, Cout, stride};
    const long long M = (long long)B * sh.OH * sh.OW;
    return gemm(FwdA{in, sh}, FwdB{w}, EpAct{out, bias, Cout}, M, Cout, 9 * Cin, 1, st);
}

cudaError_t cnn_conv_backward(const __nv_bfloat16 *in, const __nv_bfloat16 *w, const __nv_bfloat16 *out,
                              const __nv_bfloat16 *gout, __nv_bfloat16 *gin, float *gw, float *gb, int B,
                              int IH, int IW, int Cin, int Cout, int stride, cudaStream_t st)
{
    ConvShape sh{B, IH, IW, Cin, (IH - 1) / stride + 1, (IW - 1) / stride + 1, Cout, stride};
    const long long Mo = (long long)B * sh.OH * sh.OW, Mi = (long long)B * IH * IW;
    cudaError_t e;
    if (gin && (e = gemm(BwdA{gout, out, sh}, BwdB{w, sh}, EpStore{gin, Cin}, Mi, Cin, 9 * Cout, 1, st)) != cudaSuccess)
        return e;
    // weight gradient: K = all output positions, split for parallelism
    const int split = (int)((Mo + 4095) / 4096);
    if ((e = gemm(WgA{gout, out, Cout}, WgB{in, sh}, EpAdd{gw, 9 * Cin}, Cout, 9 * Cin, (int)Mo,
                  split > 0 ? split : 1, st)) != cudaSuccess)
        return e;
    dim3 grid(64, (unsigned)Cout);
    k_bias_grad<<<grid, 256, 0, st>>>(gout, out, Mo, Cout, gb);
    return cudaGetLastError();
}

cudaError_t cnn_input(const float *y, const float *s, const uint8_t *valid, const int32_t *desc, int first,
                      int count, int64_t n_pix, __nv_bfloat16 *img, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    k_cnn_input<<<(unsigned)count, 256, 0, st>>>(y, s, valid, desc, first, (long long)n_pix, img);
    return cudaGetLastError();
}

cudaError_t cnn_head_forward(const __nv_bfloat16 *act, int B, int P, int C, const float *wl,
                             const float *bl, int J, float *pooled, float *out, cudaStream_t st)
{
    k_head_forward<<<(unsigned)B, 128, 0, st>>>(act, P, C, wl, bl, J, pooled, out);
    return cudaGetLastError();
}

cudaError_t cnn_head_backward(const float *out, const float *target, int B, int J, const float *pooled,
                              const float *wl, int C, int P, float *gwl, float *gbl, __nv_bfloat16 *gact,
                              float *loss, cudaStream_t st)
{
    k_head_backward<<<(unsigned)B, 128, 0, st>>>(out, target, B, J, pooled, wl, C, P, gwl, gbl, gact, loss);
    return cudaGetLastError();
}

cudaError_t cnn_adam(float *w, const float *gw, float *m1, float *m2, long long n, float lr, int step,
                     __nv_bfloat16 *wb, cudaStream_t st)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<256, 256, 0, st>>>(w, gw, m1, m2, n, lr, b1, b2, 1e-8f, c1, c2, wb);
    return cudaGetLastError();
}

cudaError_t cnn_propose_trial(const double *poses, const float *out, int n, const double scale[6], double *trial,
                              cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_propose_trial<<<(6 * n + 255) / 256, 256, 0, st>>>(poses, out, n, scale[0], scale[1], scale[2], scale[3],
                                                          scale[4], scale[5], trial);
    return cudaGetLastError();
}

cudaError_t cnn_propose_select(const double *ncc0, const double *ncc1, const double *trial, int n, double *poses,
                               int32_t *accepted, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_propose_select<<<(n + 255) / 256, 256, 0, st>>>(ncc0, ncc1, trial, n, poses, accepted);
    return cudaGetLastError();
}

cudaError_t cnn_to_bf16(const float *a, __nv_bfloat16 *b, long long n, cudaStream_t st)
{
    k_to_bf16<<<256, 256, 0, st>>>(a, b, n);
    return cudaGetLastError();
}

}  // namespace pvr
