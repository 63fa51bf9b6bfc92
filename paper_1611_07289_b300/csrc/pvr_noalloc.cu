// pvr_simulate_noalloc: the forward model for callers that cannot allocate
// device memory.
//
// The regular entry points take their scratch (the per-patch fixed-point
// sample table, the device copy of the geometry, the error word) from a
// pvr_ctx, and creating a context calls cudaMalloc.  Some callers cannot do
// that: a host application that hands all device memory to its own pool
// allocator and forbids other allocations, or a latency-bound loop where an
// allocation (which may synchronise the device) is not acceptable after
// start-up.  This file gives them one context-free variant of pvr_simulate
// whose scratch is a file-scope device array: every GPU that loads the
// library carries it until the process exits, and no call allocates.
//
// Limits: at most kNoAllocMaxPatches patches per call; the geometry and
// PSF / pose settings pass the same checks as in pvr_ctx_create.  All calls
// share the one array, so calls that overlap on the GPU (different streams,
// or different host threads on the same device) race; serialise them.  The
// first call on a device looks up the array's device address
// (cudaGetSymbolAddress) once, with that device current -- make that first
// call before starting any stream capture.  Problems only the device sees
// (a malformed patch row, a non-finite pose) set the array's error word,
// which stays set over later calls until pvr_noalloc_status reads and
// clears it.
#include <math.h>
#include <string.h>

#include <mutex>

#include "pvr_internal.h"

namespace pvr {
namespace {

constexpr int kNoAllocMaxPatches = 8192;
constexpr size_t kGeomBytes = (sizeof(DevGeom) + 255) / 256 * 256;
constexpr size_t kFixBytes = (size_t)kNoAllocMaxPatches * kFixStride * sizeof(int32_t);
constexpr size_t kErrOffset = kGeomBytes + kFixBytes;
constexpr size_t kScratchBytes = kErrOffset + 256;

// The scratch itself: [geometry | fixed-point table | error word].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host view of the scratch, one device address per device (looked up once).
constexpr int kMaxDevices = 64;
std::mutex g_lock;
unsigned char *g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (null on failure).
unsigned char *scratch_base()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_lock);
    if (!g_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return nullptr;
        g_addr[dev] = (unsigned char *)ptr;
    }
    return g_addr[dev];
}

// Store the geometry (a kernel parameter) into the scratch, stream-ordered.
__global__ void k_store_geometry(DevGeom g, unsigned char *dst)
{
    *reinterpret_cast<DevGeom *>(dst) = g;
}

}  // namespace
}  // namespace pvr

using namespace pvr;

extern "C" PVR_API int pvr_simulate_noalloc(const pvr_geometry *geom, const pvr_params *prm,
                                            const float *x, const pvr_patches *pp,
                                            const double *poses, float *sim, uint8_t *valid,
                                            void *stream)
{
    if (!geom || !prm || !pp) return PVR_ERR_INVALID_ARG;
    if (pp->n < 0 || pp->n > kNoAllocMaxPatches) return PVR_ERR_INVALID_ARG;
    if (pp->n == 0) return PVR_OK;
    if (!pp->desc || !x || !poses || !sim || !valid) return PVR_ERR_INVALID_ARG;
    const pvr_geometry *g = geom;
    if (validate_setup(g, prm)) return PVR_ERR_INVALID_ARG;
    int max_side = pp->max_side > 0 ? pp->max_side : prm->max_patch_side;
    if (max_side < 1 || max_side > 256 || pp->n_pix < 1 || pp->n_pix >= ((int64_t)1 << 31))
        return PVR_ERR_INVALID_ARG;
    unsigned char *base = scratch_base();
    if (!base) return PVR_ERR_CUDA;

    // geometry and PSF tables, as pvr_ctx_create derives them
    DevGeom hg;
    memset(&hg, 0, sizeof hg);
    hg.nx = g->nx;
    hg.ny = g->ny;
    hg.nz = g->nz;
    hg.n_stacks = g->n_stacks;
    long long off = 0;
    for (int s = 0; s < g->n_stacks; ++s) {
        hg.sw[s] = g->stack_w[s];
        hg.sh[s] = g->stack_h[s];
        hg.sk[s] = g->stack_k[s];
        hg.stack_off[s] = off;
        off += (long long)g->stack_w[s] * g->stack_h[s] * g->stack_k[s];
        memcpy(hg.p2w[s], g->pixel_to_world[s], 12 * sizeof(double));
    }
    memcpy(hg.w2v, g->world_to_voxel, 12 * sizeof(double));
    hg.dz = prm->psf_dz;
    PsfTab t;
    make_psf_tab(g, prm, &t);

    cudaStream_t st = (cudaStream_t)stream;
    DevGeom *d_geom = reinterpret_cast<DevGeom *>(base);
    int32_t *d_fix = reinterpret_cast<int32_t *>(base + kGeomBytes);
    int32_t *d_err = reinterpret_cast<int32_t *>(base + kErrOffset);
    // every call rewrites the geometry and the table rows it uses; the error
    // word is sticky (zero when the library loads, cleared by
    // pvr_noalloc_status)
    k_store_geometry<<<1, 1, 0, st>>>(hg, base);
    if (cudaGetLastError() != cudaSuccess) return PVR_ERR_CUDA;
    if (launch_pose_to_fixed(d_geom, pp->desc, poses, prm->n_params, pp->n, pp->n_pix, max_side, t.kxy, t.kz,
                             d_fix, d_err, st) != cudaSuccess)
        return PVR_ERR_CUDA;
    Tiling tl;
    tl.T = max_side <= 64 ? max_side : 64;
    tl.tiles_x = tl.tiles_y = (max_side + tl.T - 1) / tl.T;
    tl.tpp = tl.tiles_x * tl.tiles_y;
    tl.member = pp->member;
    if (launch_simulate(d_geom, t, tl, g->nx, g->ny, g->nz, x, nullptr, pp->desc, d_fix, pp->n, nullptr, sim,
                        valid, nullptr, st) != cudaSuccess)
        return PVR_ERR_CUDA;
    return PVR_OK;
}

extern "C" PVR_API int pvr_noalloc_status(void *stream)
{
    unsigned char *base = scratch_base();
    if (!base) return PVR_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *d_err = reinterpret_cast<int32_t *>(base + kErrOffset);
    int32_t h = 0;
    if (cudaMemcpyAsync(&h, d_err, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess) return PVR_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PVR_ERR_CUDA;
    if (h != 0 && cudaMemsetAsync(d_err, 0, sizeof h, st) != cudaSuccess) return PVR_ERR_CUDA;
    if (h & 1) return PVR_ERR_BOUNDS;
    if (h & 2) return PVR_ERR_NUMERIC;
    return PVR_OK;
}
