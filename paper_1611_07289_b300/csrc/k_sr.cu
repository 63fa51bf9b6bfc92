// Edge-preserving diffusion step of the regularised super-resolution update
// (the anisotropic-diffusion regularisation of the SR framework PVR builds
// on, Sec. I / Sec. II; the paper prints no formula, this is the reading the
// oracle's or_sr_update states).  After the SIRT step has left u in the
// volume, every voxel v that the data reached (conf > conf_eps) becomes
//   max(u(v) + lambda * sum_d w_d psi(u(v + d) - u(v)), 0),
//   psi(D) = D / sqrt(1 + (D / delta)^2),  w_d = (1 / |d|^2) / (44 / 3),
// over its 26 neighbours d inside the volume; the others keep u(v).
//
// One CTA per 32 x 8 x 4 block of voxels.  The block and a one-voxel halo
// (the x range widened to 40 so that the box starts on a 16-byte boundary)
// are staged in shared memory by one TMA tiled load (cp.async.bulk.tensor.3d
// with mbarrier completion; samples outside the volume arrive as zeros and
// are never used), or by plain loads when the volume's row pitch rules TMA
// out.  The result goes to a separate volume (neighbouring blocks read the
// old values as halo); the accumulator is read and cleared at each thread's
// own voxel only, so no block clears data another still needs.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <mutex>

#include "pvr_internal.h"

namespace pvr {
namespace {

constexpr int kBX = 32, kBY = 8, kBZ = 4;                          // voxels per block
constexpr int kHX = 4;                                             // x halo: 16-byte aligned box start
constexpr int kSX = kBX + 2 * kHX, kSY = kBY + 2, kSZ = kBZ + 2;   // staged box 40 x 10 x 6
constexpr unsigned kBoxBytes = kSX * kSY * kSZ * 4;
constexpr unsigned kWaitPolls = 1u << 24;

// Conf of voxel v (then cleared) from interleaved (addon, conf) pairs ...
struct AccPairs {
    float2 *acc;
    __device__ float take(size_t v) const
    {
        const float c = acc[v].y;
        acc[v] = make_float2(0.f, 0.f);
        return c;
    }
};

// ... or from separate arrays (cleared when asked).
struct AccSplit {
    float *addon, *conf;
    int clear;
    __device__ float take(size_t v) const
    {
        const float c = conf[v];
        if (clear) {
            addon[v] = 0.f;
            conf[v] = 0.f;
        }
        return c;
    }
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity)
{
    for (unsigned i = 0; i < kWaitPolls; ++i) {
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

// Flux sum of one voxel from the staged box; INNER: every neighbour is
// inside the volume (no bounds tests).
template <bool INNER>
__device__ __forceinline__ float box_flux(const float (&box)[kSZ][kSY][kSX], int cx, int cy, int cz, int gx, int gy,
                                          int gz, int nx, int ny, int nz, float c, float inv_delta)
{
    const float W = 6.f + 12.f / 2.f + 8.f / 3.f;
    const float w1 = 1.f / W, w2 = (1.f / 2.f) / W, w3 = (1.f / 3.f) / W;
    float flux = 0.f;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int r2 = dx * dx + dy * dy + dz * dz;
                if (r2 == 0) continue;
                if (!INNER) {
                    const int qx = gx + dx, qy = gy + dy, qz = gz + dz;
                    if (qx < 0 || qy < 0 || qz < 0 || qx >= nx || qy >= ny || qz >= nz) continue;
                }
                const float D = box[cz + 1 + dz][cy + 1 + dy][cx + kHX + dx] - c;
                const float t = D * inv_delta;
                const float psi = D * rsqrtf(fmaf(t, t, 1.f));
                flux = fmaf(r2 == 1 ? w1 : (r2 == 2 ? w2 : w3), psi, flux);
            }
    return flux;
}

constexpr int kPerThread = kBX * kBY * kBZ / 256;   // voxels per thread (blocks of 256 threads)

template <bool TMA, class ACC>
__global__ void __launch_bounds__(256) k_sr_diffuse(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ u,
                                                    ACC acc, float *__restrict__ xo, int nx, int ny, int nz,
                                                    float lambda, float inv_delta, float conf_eps,
                                                    int32_t *__restrict__ err)
{
    __shared__ __align__(128) float box[kSZ][kSY][kSX];
    __shared__ __align__(8) uint64_t bar;
    const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * kBY, z0 = blockIdx.z * kBZ;
    if (TMA && threadIdx.x == 0) {
        const uint32_t b = smem_u32(&bar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(kBoxBytes) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
            "%4}], [%5];" ::"r"(smem_u32(&box[0][0][0])),
            "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(x0 - kHX), "r"(y0 - 1), "r"(z0 - 1), "r"(b)
            : "memory");
    }
    // each thread's voxels and their accumulator entries, read (and
    // cleared) while the tile is in flight
    float conf[kPerThread];
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        const int k = threadIdx.x + 256 * j;
        const int gx = x0 + k % kBX, gy = y0 + (k / kBX) % kBY, gz = z0 + k / (kBX * kBY);
        conf[j] = (gx < nx && gy < ny && gz < nz) ? acc.take(((size_t)gz * ny + gy) * nx + gx) : 0.f;
    }
    if (TMA) {
        __syncthreads();   // the barrier is initialised before anyone waits on it
        if (!bar_wait(smem_u32(&bar), 0)) {
            // give up: report, then wait once more (bounded) for the copy in flight
            if (threadIdx.x == 0) atomicOr(err, 4);
            bar_wait(smem_u32(&bar), 0);
            return;
        }
    } else {
        for (int i = threadIdx.x; i < kSX * kSY * kSZ; i += blockDim.x) {
            const int lx = i % kSX, ly = (i / kSX) % kSY, lz = i / (kSX * kSY);
            const int gx = x0 - kHX + lx, gy = y0 - 1 + ly, gz = z0 - 1 + lz;
            const bool in = gx >= 0 && gy >= 0 && gz >= 0 && gx < nx && gy < ny && gz < nz;
            box[lz][ly][lx] = in ? __ldg(u + ((size_t)gz * ny + gy) * nx + gx) : 0.f;
        }
        __syncthreads();
    }
    // blocks whose one-voxel shell lies inside the volume need no bounds tests
    const bool inner = x0 >= 1 && y0 >= 1 && z0 >= 1 && x0 + kBX < nx && y0 + kBY < ny && z0 + kBZ < nz;
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        const int k = threadIdx.x + 256 * j;
        const int cx = k % kBX, cy = (k / kBX) % kBY, cz = k / (kBX * kBY);
        const int gx = x0 + cx, gy = y0 + cy, gz = z0 + cz;
        if (gx >= nx || gy >= ny || gz >= nz) continue;
        const float c = box[cz + 1][cy + 1][cx + kHX];
        float out = c;
        if (conf[j] > conf_eps) {
            const float flux = inner ? box_flux<true>(box, cx, cy, cz, gx, gy, gz, nx, ny, nz, c, inv_delta)
                                     : box_flux<false>(box, cx, cy, cz, gx, gy, gz, nx, ny, nz, c, inv_delta);
            out = fmaxf(c + lambda * flux, 0.f);
        }
        xo[((size_t)gz * ny + gy) * nx + gx] = out;
    }
}

// cuTensorMapEncodeTiled from the driver, looked up once.
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// Tiled tensor map of the float32 volume u for the staged box, if TMA can
// address it (row pitch and base a multiple of 16 bytes).
bool volume_tensor_map(const float *u, int nx, int ny, int nz, CUtensorMap *map)
{
    if ((nx * 4) % 16 != 0 || (reinterpret_cast<uintptr_t>(u) & 15) != 0) return false;
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
    const cuuint32_t boxd[3] = {(cuuint32_t)kSX, (cuuint32_t)kSY, (cuuint32_t)kSZ};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(u), dims, strides, boxd, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class ACC>
cudaError_t diffuse(const float *u, ACC acc, float *xo, int nx, int ny, int nz, float lambda, float delta,
                    float conf_eps, int32_t *err, cudaStream_t st)
{
    const dim3 grid((unsigned)((nx + kBX - 1) / kBX), (unsigned)((ny + kBY - 1) / kBY), (unsigned)((nz + kBZ - 1) / kBZ));
    CUtensorMap map;
    memset(&map, 0, sizeof map);
    const float inv_delta = 1.f / delta;
    if (volume_tensor_map(u, nx, ny, nz, &map))
        k_sr_diffuse<true, ACC><<<grid, 256, 0, st>>>(map, u, acc, xo, nx, ny, nz, lambda, inv_delta, conf_eps, err);
    else
        k_sr_diffuse<false, ACC><<<grid, 256, 0, st>>>(map, u, acc, xo, nx, ny, nz, lambda, inv_delta, conf_eps, err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sr_diffuse_pairs(const float *u, float2 *acc, float *xo, int nx, int ny, int nz, float lambda,
                                    float delta, float conf_eps, int32_t *err, cudaStream_t st)
{
    return diffuse(u, AccPairs{acc}, xo, nx, ny, nz, lambda, delta, conf_eps, err, st);
}

cudaError_t launch_sr_diffuse_split(const float *u, float *addon, float *conf, int clear, float *xo, int nx, int ny,
                                    int nz, float lambda, float delta, float conf_eps, int32_t *err, cudaStream_t st)
{
    return diffuse(u, AccSplit{addon, conf, clear}, xo, nx, ny, nz, lambda, delta, conf_eps, err, st);
}

bool sr_diffuse_uses_tma(const float *u, int nx, int ny, int nz)
{
    CUtensorMap map;
    return volume_tensor_map(u, nx, ny, nz, &map);
}

}  // namespace pvr
