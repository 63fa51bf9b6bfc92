// Kernels of the learned pose proposal: a small 2-D CNN over (acquired
// patch, simulated patch) pairs that predicts the rigid correction of the
// patch pose.  Activations and weights are bfloat16 (NHWC, channels a
// multiple of 16), accumulation float32.
//
// Every 3x3 convolution pass is one implicit GEMM on the 5th-generation
// tensor cores (tcgen05.mma kind::f16, bf16 x bf16 -> f32, accumulator in
// tensor memory), with the im2col gather folded into the operand loads:
//   forward      C[m = (n, oy, ox)][co]       = sum_k A[m][k = (ky, kx, ci)] B[co][k]
//   input grad   C[m = (n, iy, ix)][ci]       = sum_k A[m][k = (ky, kx, co)] B[ci][k]
//   weight grad  C[(ky, kx, ci)][co]          = sum_{m = (n, oy, ox)} act[m][(ky, kx, ci)] g[m][co]
//                (transposed, with an extra row of ones whose result is
//                the bias gradient sum_m g[m][co])
// The tile loaders of the first two passes turn (row, k0) into 8
// consecutive k values (K-major operands); those of the weight gradient
// turn (row group, k) into 8 consecutive rows at one k (MN-major).
#include <cuda_bf16.h>

#include "pvr_internal.h"

namespace pvr {
namespace {

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

// ---- MN-major loaders (weight gradient): 8 consecutive rows at one k ----

// weight-grad A' (rows k9 = (ky, kx, ci), k = output position m): the 8
// input channels ci..ci+7 under tap (ky, kx) of position m, one 16-byte
// load; row 9 Cin is all ones (its GEMM row is the bias gradient), rows
// beyond it are zero
struct WgBmn {
    const __nv_bfloat16 *in;
    ConvShape sh;
    __device__ uint4 operator()(long long k9, int m, long long N, int K) const
    {
        const int K9 = 9 * sh.Cin;
        if (m >= K || k9 > K9) return zero4();
        if (k9 == K9) return make_uint4(0x3F80u, 0u, 0u, 0u);   // bf16 1.0 in row K9
        const int tap = (int)(k9 / sh.Cin), ci = (int)(k9 - (long long)tap * sh.Cin);
        const int ky = tap / 3, kx = tap - ky * 3;
        const int ox = m % sh.OW, r = m / sh.OW, oy = r % sh.OH, n = r / sh.OH;
        const int iy = oy * sh.stride + ky - 1, ix = ox * sh.stride + kx - 1;
        if (iy < 0 || ix < 0 || iy >= sh.IH || ix >= sh.IW) return zero4();
        return *reinterpret_cast<const uint4 *>(in + (((size_t)n * sh.IH + iy) * sh.IW + ix) * sh.Cin + ci);
    }
};

// weight-grad B' (rows co, k = output position m): the masked upstream
// gradient of output channels co..co+7 at position m
struct WgAmn {
    const __nv_bfloat16 *g, *out;
    int Cout;
    __device__ uint4 operator()(long long co, int m, long long N, int K) const
    {
        if (co >= N || m >= K) return zero4();
        const size_t o = (size_t)m * Cout + co;
        const uint4 gv = *reinterpret_cast<const uint4 *>(g + o), ov = *reinterpret_cast<const uint4 *>(out + o);
        const __nv_bfloat16 *gp = reinterpret_cast<const __nv_bfloat16 *>(&gv);
        const __nv_bfloat16 *op = reinterpret_cast<const __nv_bfloat16 *>(&ov);
        const __nv_bfloat16 zero = __float2bfloat16(0.f);
        unsigned u[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            u[j] = pack2(__bfloat162float(op[2 * j]) > 0.f ? gp[2 * j] : zero,
                         __bfloat162float(op[2 * j + 1]) > 0.f ? gp[2 * j + 1] : zero);
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

// float32 accumulation of split-K partial sums into the weight gradient
// gw[co][k9], computed transposed (GEMM row m = k9, column n = co); GEMM
// row K9 is the bias gradient gb[co]
struct EpAddT {
    float *out, *bias;
    int K9;
    __device__ void operator()(long long m, long long n, float v) const
    {
        if (m < K9)
            atomicAdd(out + (size_t)n * K9 + m, v);
        else if (m == K9)
            atomicAdd(bias + n, v);
    }
};

// ---- tcgen05 implicit GEMM ----
//
// One CTA (4 warps) computes a 128 x BN tile of C = A B^T (A: M x K, B:
// N x K, BN = N <= 64, a multiple of 16), each operand K-major (16-byte
// chunks of 8 consecutive k) or MN-major (chunks of 8 consecutive rows at
// one k: the weight gradient, whose k -- the output position -- is not the
// contiguous dimension of either operand).  K advances in
// stages of kTK = 32: all 128 threads gather the stage's A rows and B rows
// through the loader functors (8 consecutive k per 16-byte chunk) into
// shared memory in the tensor core's canonical no-swizzle K-major layout --
// 8-row x 16-byte core matrices of 128 contiguous bytes, the 4 core
// matrices of a row group side by side along K (leading-dimension offset
// 128 B), row groups 512 B apart (stride-dimension offset) -- then one
// thread issues the stage's two m128 x nBN x k16 MMAs, which accumulate in
// tensor memory (128 lanes x BN float32 columns), and commits them to the
// stage buffer's mbarrier.  Two buffers: the gather of stage s + 1 overlaps
// the MMAs of stage s.  The epilogue reads the accumulator back with
// tcgen05.ld (warp w owns rows 32w..32w+31) and hands each value to EP.
// Every wait is bounded: on expiry the kernel records PVR_ERR_TIMEOUT in the
// device word read by pvr_net_status, skips the rest and still frees its
// tensor memory.
constexpr int kTM = 128, kTK = 32;
constexpr int kStageA = kTM * kTK * 2, kStageB = 64 * kTK * 2;   // bytes per stage buffer
constexpr unsigned kWaitLimit = 1u << 24;                         // polls of one bounded wait

__device__ unsigned g_tc_err;   // 1: a bounded wait of the tensor-core GEMM expired

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05 format): start address, leading-
// and stride-dimension byte offsets (all >> 4), descriptor version 1, no
// swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: f32 accumulator, bf16 A and B,
// each K-major or MN-major, shape M x N.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N, bool mn_a, bool mn_b)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((mn_a ? 1u : 0u) << 15) | ((mn_b ? 1u : 0u) << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (unsigned i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Canonical K-major offset (bytes) of the 16-byte chunk of row r, k-chunk kc.
__device__ __forceinline__ uint32_t canon_off(int r, int kc) { return (uint32_t)((r >> 3) * 512 + kc * 128 + (r & 7) * 16); }

// Canonical MN-major offset (bytes) of the 16-byte chunk holding rows
// 8g..8g+7 at k index p: core matrices of 8 k-rows x 8 elements, the 4
// k-groups of a row group 128 B apart, row groups 512 B apart -- the same
// extents as the K-major tiles.
__device__ __forceinline__ uint32_t canon_off_mn(int g, int p) { return (uint32_t)(g * 512 + (p >> 3) * 128 + (p & 7) * 16); }

template <int BN, bool MNA, bool MNB, class LA, class LB, class EP>
__global__ void __launch_bounds__(128) k_gemm_tc(LA la, LB lb, EP ep, long long M, long long N, int K,
                                                 int k_per_split)
{
    __shared__ __align__(1024) unsigned char As[2][kStageA];
    __shared__ __align__(1024) unsigned char Bs[2][kStageB];
    __shared__ __align__(8) uint64_t mma_bar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    constexpr int kCols = BN < 32 ? 32 : BN;   // tensor-memory columns (power of 2, >= 32)
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long m0 = (long long)blockIdx.x * kTM;
    const int kb = blockIdx.z * k_per_split;
    const int ke = min(K, kb + k_per_split);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    constexpr uint32_t idesc = umma_idesc(kTM, BN, MNA, MNB);
    int stage = 0;
    for (int k = kb; k < ke; k += kTK, ++stage) {
        const int b = stage & 1;
        // the MMAs that read this buffer two stages ago must be done
        if (stage >= 2 && !mbar_wait(smem_u32(&mma_bar[b]), (uint32_t)(((stage >> 1) - 1) & 1))) abort_flag = 1;
        if (MNA) {
            // chunk = 8 consecutive rows (row group g) at one k: consecutive
            // threads take consecutive k, one 16-byte core-matrix row each
            for (int c = tid; c < kTM * (kTK / 8); c += 128) {
                const int p = c % kTK, g = c / kTK;
                *reinterpret_cast<uint4 *>(As[b] + canon_off_mn(g, p)) = la(m0 + 8 * g, k + p, M, ke);
            }
        } else {
            for (int c = tid; c < kTM * (kTK / 8); c += 128) {
                const int r = c & (kTM - 1), kc = c / kTM;
                *reinterpret_cast<uint4 *>(As[b] + canon_off(r, kc)) = la(m0 + r, k + 8 * kc, M, ke);
            }
        }
        if (MNB) {
            for (int c = tid; c < BN * (kTK / 8); c += 128) {
                const int p = c % kTK, g = c / kTK;
                *reinterpret_cast<uint4 *>(Bs[b] + canon_off_mn(g, p)) = lb(8 * g, k + p, N, ke);
            }
        } else {
            for (int c = tid; c < BN * (kTK / 8); c += 128) {
                const int r = c % BN, kc = c / BN;
                *reinterpret_cast<uint4 *>(Bs[b] + canon_off(r, kc)) = lb(r, k + 8 * kc, N, ke);
            }
        }
        // generic-proxy stores become visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (abort_flag) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(As[b]), b0 = smem_u32(Bs[b]);
#pragma unroll
            for (int j = 0; j < kTK / 16; ++j) {
                const uint64_t ad = umma_desc(a0 + 256 * j, 128, 512), bd = umma_desc(b0 + 256 * j, 128, 512);
                const uint32_t acc = (k > kb || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mma_bar[b]))
                         : "memory");
        }
    }
    // the last stage's commit covers every MMA issued before it
    if (stage > 0 && !abort_flag && !mbar_wait(smem_u32(&mma_bar[(stage - 1) & 1]), (uint32_t)(((stage - 1) >> 1) & 1)))
        abort_flag = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (abort_flag) {
        if (tid == 0) atomicOr(&g_tc_err, 1u);
    } else if (stage > 0) {
        const long long row = m0 + warp * 32 + (tid & 31);
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M)
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (c0 + i < N) ep(row, (long long)(c0 + i), __uint_as_float(v[i]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
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

// Head: out[b][j] = bias[j] + sum_f wl[j][f] feat[b][f] over the F = P C
// features of the last activation (B x P x C, flattened in its NHWC order,
// so the head sees where in the patch each feature lies), float32.  One CTA
// of 128 threads per sample; feat receives the features as float32 for the
// backward pass.  J <= 8.
__global__ void __launch_bounds__(128) k_head_forward(const __nv_bfloat16 *__restrict__ act, int F,
                                                      const float *__restrict__ wl, const float *__restrict__ bl,
                                                      int J, float *__restrict__ feat, float *__restrict__ out)
{
    __shared__ float red[4][8];
    const int b = blockIdx.x, t = threadIdx.x;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int f = t; f < F; f += blockDim.x) {
        const float v = __bfloat162float(act[(size_t)b * F + f]);
        feat[(size_t)b * F + f] = v;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < J) acc[j] = fmaf(wl[(size_t)j * F + f], v, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
    if ((t & 31) == 0)
#pragma unroll
        for (int j = 0; j < 8; ++j) red[t >> 5][j] = acc[j];
    __syncthreads();
    if (t < J) out[(size_t)b * J + t] = bl[t] + red[0][t] + red[1][t] + red[2][t] + red[3][t];
}

// Head backward for the loss mean_b sum_j (out - target)^2 / B: gradients
// of the linear layer (accumulated into gwl, gbl) and of the last
// activation (bf16).  One CTA of 128 threads per sample.
__global__ void __launch_bounds__(128) k_head_backward(const float *__restrict__ out,
                                                       const float *__restrict__ target, int B, int J,
                                                       const float *__restrict__ feat, const float *__restrict__ wl,
                                                       int F, float *__restrict__ gwl, float *__restrict__ gbl,
                                                       __nv_bfloat16 *__restrict__ gact, float *__restrict__ loss)
{
    __shared__ float go[8];
    const int b = blockIdx.x, t = threadIdx.x;
    if (t < J) {
        const float e = out[(size_t)b * J + t] - target[(size_t)b * J + t];
        go[t] = 2.f * e / B;
        atomicAdd(loss, e * e / B);
        atomicAdd(gbl + t, go[t]);
    }
    __syncthreads();
    for (int f = t; f < F; f += blockDim.x) {
        const float v = feat[(size_t)b * F + f];
        float ga = 0.f;
        for (int j = 0; j < J; ++j) {
            ga = fmaf(wl[(size_t)j * F + f], go[j], ga);
            atomicAdd(gwl + (size_t)j * F + f, go[j] * v);
        }
        gact[(size_t)b * F + f] = __float2bfloat16(ga);
    }
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

// trial = pose + (S t, S w): the network's correction of patch p is given
// in the frame of its stack -- translation t and rotation angles w along /
// about the column, row and slice-normal directions, out[p][k] times
// scale[k] -- and S = the unit column, row and normal vectors of the
// stack's pixel-to-world map maps both to world pose increments (mm, and
// degrees about the world axes, to first order in the angles).
__global__ void k_propose_trial(const DevGeom *__restrict__ g, const int32_t *__restrict__ desc,
                                const double *__restrict__ poses, const float *__restrict__ out, int n,
                                double s0, double s1, double s2, double s3, double s4, double s5,
                                double *__restrict__ trial)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double *P = g->p2w[desc[8 * (size_t)p]];
    double S[3][3];   // S[r][c]: component r of unit axis c
    for (int c = 0; c < 3; ++c) {
        const double nr = sqrt(P[c] * P[c] + P[4 + c] * P[4 + c] + P[8 + c] * P[8 + c]);
        for (int r = 0; r < 3; ++r) S[r][c] = nr > 0.0 ? P[4 * r + c] / nr : 0.0;
    }
    const double sc[6] = {s0, s1, s2, s3, s4, s5};
    double loc[6];
    for (int k = 0; k < 6; ++k) loc[k] = sc[k] * (double)out[6 * (size_t)p + k];
    for (int r = 0; r < 3; ++r) {
        double dt = 0.0, dw = 0.0;
        for (int c = 0; c < 3; ++c) {
            dt += S[r][c] * loc[c];
            dw += S[r][c] * loc[3 + c];
        }
        trial[6 * (size_t)p + r] = poses[6 * (size_t)p + r] + dt;
        trial[6 * (size_t)p + 3 + r] = poses[6 * (size_t)p + 3 + r] + dw;
    }
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

// C (+)= A B^T on the tensor cores; N <= 64.  split > 1 cuts K into slices
// (blockIdx.z) whose partial sums the epilogue adds.
template <bool MNA = false, bool MNB = false, class LA, class LB, class EP>
cudaError_t gemm(LA la, LB lb, EP ep, long long M, long long N, int K, int split, cudaStream_t st)
{
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (N > 64) return cudaErrorInvalidValue;
    int kps = (K + split - 1) / split;
    kps = (kps + kTK - 1) / kTK * kTK;
    const int nz = (K + kps - 1) / kps;
    dim3 grid((unsigned)((M + kTM - 1) / kTM), 1, (unsigned)nz);
    if (N <= 16)
        k_gemm_tc<16, MNA, MNB, LA, LB, EP><<<grid, 128, 0, st>>>(la, lb, ep, M, N, K, kps);
    else if (N <= 32)
        k_gemm_tc<32, MNA, MNB, LA, LB, EP><<<grid, 128, 0, st>>>(la, lb, ep, M, N, K, kps);
    else
        k_gemm_tc<64, MNA, MNB, LA, LB, EP><<<grid, 128, 0, st>>>(la, lb, ep, M, N, K, kps);
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
    // weight and bias gradient in one GEMM, transposed so that the 128-row
    // tile runs over the 9 Cin (tap, input channel) pairs plus a row of ones
    // (the bias): rows k9, columns co, K = all output positions (MN-major
    // operands), split for parallelism
    const int split = (int)((Mo + 4095) / 4096);
    return gemm<true, true>(WgBmn{in, sh}, WgAmn{gout, out, Cout}, EpAddT{gw, gb, 9 * Cin}, 9 * Cin + 1, Cout,
                            (int)Mo, split > 0 ? split : 1, st);
}

cudaError_t cnn_input(const float *y, const float *s, const uint8_t *valid, const int32_t *desc, int first,
                      int count, int64_t n_pix, __nv_bfloat16 *img, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    k_cnn_input<<<(unsigned)count, 256, 0, st>>>(y, s, valid, desc, first, (long long)n_pix, img);
    return cudaGetLastError();
}

cudaError_t cnn_head_forward(const __nv_bfloat16 *act, int B, int F, const float *wl, const float *bl, int J,
                             float *feat, float *out, cudaStream_t st)
{
    if (J > 8) return cudaErrorInvalidValue;
    k_head_forward<<<(unsigned)B, 128, 0, st>>>(act, F, wl, bl, J, feat, out);
    return cudaGetLastError();
}

cudaError_t cnn_head_backward(const float *out, const float *target, int B, int J, const float *feat,
                              const float *wl, int F, float *gwl, float *gbl, __nv_bfloat16 *gact, float *loss,
                              cudaStream_t st)
{
    if (J > 8) return cudaErrorInvalidValue;
    k_head_backward<<<(unsigned)B, 128, 0, st>>>(out, target, B, J, feat, wl, F, gwl, gbl, gact, loss);
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

cudaError_t cnn_propose_trial(const DevGeom *g, const int32_t *desc, const double *poses, const float *out, int n,
                              const double scale[6], double *trial, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_propose_trial<<<(n + 127) / 128, 128, 0, st>>>(g, desc, poses, out, n, scale[0], scale[1], scale[2], scale[3],
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

// Read and clear the timeout word of the tensor-core GEMM (stream-ordered
// copy into *host_flag; the caller synchronises).
cudaError_t cnn_read_timeout(unsigned *host_flag, cudaStream_t st)
{
    void *word = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&word, g_tc_err);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(host_flag, word, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    return cudaMemsetAsync(word, 0, sizeof(unsigned), st);
}

}  // namespace pvr
