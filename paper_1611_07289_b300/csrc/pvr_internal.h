// Internal declarations of libpvr (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pvr.h"

namespace pvr {

constexpr int kFracBits = 20;              // Q11.20 sample coordinates
constexpr int kFixStride = 16;             // int32 per patch in the fixed table
constexpr int kPartStride = 8;             // float64 per (patch, tile) partial slot
constexpr int kGradStride = 16;            // float64 per (patch, tile) gradient-moment slot
constexpr int kRegStride = 12;             // float64 per patch pose slot

// Geometry as the kernels read it (device memory, copied at context creation).
struct DevGeom {
    int nx, ny, nz, n_stacks;
    int sw[PVR_MAX_STACKS], sh[PVR_MAX_STACKS], sk[PVR_MAX_STACKS];
    long long stack_off[PVR_MAX_STACKS];   // element offset of stack s in the packed buffer
    double w2v[12];
    double p2w[PVR_MAX_STACKS][12];
    double dz;                             // through-plane PSF step, mm
};

// PSF weight tables (float32), passed to kernels by value.
struct PsfTab {
    int kxy, kz;
    float gxy[2 * PVR_MAX_KXY + 1];
    float gz[PVR_MAX_STACKS][2 * PVR_MAX_KZ + 1];
};

// PSF tables of a geometry and parameter set (Gaussian or Taylor-sinc
// in-plane profile, Gaussian slice profile).
void make_psf_tab(const pvr_geometry *g, const pvr_params *prm, PsfTab *tab);

// Geometry and PSF / pose-parameter checks shared by pvr_ctx_create and the
// context-free forward model: null when valid, else a one-line reason.
const char *validate_setup(const pvr_geometry *g, const pvr_params *prm);

// Pose parameter count (6 or 12) and device geometry of a context.
int ctx_n_params(const pvr_ctx *c);
const DevGeom *ctx_dev_geom(const pvr_ctx *c);

// Patch-tile decomposition shared by the per-patch kernels: tile side T
// pixels, tiles_x * tiles_y tiles per patch (the largest patch's count);
// block b works on patch b / tpp, tile b % tpp.
struct Tiling {
    int T;
    int tiles_x, tiles_y, tpp;
    const uint8_t *member = nullptr;   // per patch pixel: 1 = part of the patch (null: all)
    // patch launch order (a permutation of 0 .. n - 1): launch position k
    // (the k-th CTA, or the k-th tile a persistent kernel takes) processes
    // tile k % tpp of patch order[k / tpp] (null: slot order)
    const int32_t *order = nullptr;
};

// Persistent work queue over the non-empty (patch, tile) slots of a patch
// table: items = slot indices (patch * tpp + tile), largest tiles first;
// counter: one device int, reset by the launcher before every launch.
struct WorkQueue {
    const int32_t *items = nullptr;
    int n_items = 0;
    int *counter = nullptr;
};

// Forward model at the best pose, kept by the registration for one-tile
// patches so that the first super-resolution pass of the same iteration
// need not simulate again: residual e = y - s, valid flag and the EM tile
// partials {N, sum e^2, min e, max e}, as the forward-model kernel writes
// them.  mode 0: off; 1: every evaluated tile (the first evaluation, at the
// starting pose); 2: tiles whose NCC improves on nbest (the registration's
// acceptance rule; every tile with fixed steps).
struct BestSim {
    float *e = nullptr;
    uint8_t *valid = nullptr;
    double *part = nullptr;
    const double *nbest = nullptr;
    int mode = 0;
    int fixed = 0;
    // a registration evaluation after the first: the gradient is needed
    // only where the trial is accepted (a rejected trial's next step uses
    // the gradient at the best pose), so one-tile patches skip the gradient
    // pass elsewhere (their gradient slots read as zero)
    int grad_if_accepted = 0;
};

// Launchers (each returns cudaGetLastError() of its launches).
// poses: float64 [n][n_params], n_params 6 (rigid) or 12 (affine).
cudaError_t launch_pose_to_fixed(const DevGeom *g, const int32_t *desc, const double *poses,
                                 int n_params, int n, int64_t n_pix, int max_side, int kxy, int kz,
                                 int32_t *fix, int32_t *err, cudaStream_t st);

// Forward model from x (quad == null) or from the quad copy of x.
cudaError_t launch_simulate(const DevGeom *g, const PsfTab &psf, const Tiling &tl, int nx, int ny,
                            int nz, const float *x, const float4 *quad, const int32_t *desc,
                            const int32_t *fix, int n, const float *y, float *sim_or_e,
                            uint8_t *valid, double *part, cudaStream_t st,
                            const WorkQueue *wq = nullptr);

// Quad copy of the volume (nx * ny * nz < 2^31): quad[i] = (x[i], x[i + 1],
// x[i + nx], x[i + nx + 1]), read by the gathers as two 16-byte loads per cell.
cudaError_t launch_build_quad(const float *x, float4 *quad, int nx, int ny, int nz, cudaStream_t st);

// pair = 1: addon points to interleaved (addon, conf) float2 pairs, conf unused.
// patch_weight (float per patch, may be null) multiplies r, not w.
cudaError_t launch_adjoint(const PsfTab &psf, const Tiling &tl, int nx, int ny, int nz,
                           const int32_t *desc, const int32_t *fix, int n, const float *r,
                           const float *w, const uint8_t *patch_mask, float *addon, float *conf,
                           int pair, cudaStream_t st, const WorkQueue *wq = nullptr,
                           const float *patch_weight = nullptr);

// Weighted SIRT step on interleaved (addon, conf) pairs; optionally clears them.
cudaError_t launch_volume_update_pairs(float *x, float2 *acc, int64_t nvox, float alpha,
                                       float conf_eps, int clear, int init_mode, cudaStream_t st);

// Copy (or add, accumulate = 1) interleaved pairs into separate arrays (either may be null).
cudaError_t launch_split_pairs(const float2 *acc, int64_t nvox, float *addon, float *conf,
                               int accumulate, cudaStream_t st);

cudaError_t launch_volume_update(float *x, float *addon, float *conf, int64_t nvox, float alpha,
                                 float conf_eps, int clear, int init_mode, cudaStream_t st);

// Edge-preserving diffusion step after the SIRT step (u = the SIRT result):
// xo = the regularised volume; the accumulator (interleaved pairs, or
// separate arrays cleared when `clear`) is read and cleared voxel by voxel.
// A bounded wait that expires sets bit 4 of the device error word.
cudaError_t launch_sr_diffuse_pairs(const float *u, float2 *acc, float *xo, int nx, int ny, int nz, float lambda,
                                    float delta, float conf_eps, int32_t *err, cudaStream_t st);
cudaError_t launch_sr_diffuse_split(const float *u, float *addon, float *conf, int clear, float *xo, int nx, int ny,
                                    int nz, float lambda, float delta, float conf_eps, int32_t *err, cudaStream_t st);
// True when the diffusion step stages its tiles by TMA for this volume.
bool sr_diffuse_uses_tma(const float *u, int nx, int ny, int nz);


// NCC moments (+ gradient when gpart != null) of every patch, gathering
// from the quad copy of the volume.  One-tile patches run one fused
// persistent kernel with a gbuf slot per CTA; otherwise the gradient pass
// streams per-lattice-point gradient sums through gbuf, in chunks of whole
// patches of at most gbuf_tiles tiles.
cudaError_t launch_ncc_grad(const DevGeom *g, const PsfTab &psf, const Tiling &tl, int nx, int ny,
                            int nz, const float *xplain, const float4 *quad, const float *y,
                            const int32_t *desc, const int32_t *fix, const double *poses, int n,
                            float *s_buf,
                            uint8_t *v_buf, double *part, double *gpart, const int32_t *active,
                            int min_valid, float *gbuf, long long gbuf_tiles, int *counter, cudaStream_t st,
                            const BestSim &bs = BestSim());
size_t ncc_gbuf_floats_per_tile(const Tiling &tl, int kxy);
// Kernel launches launch_ncc_grad makes for these arguments.
int ncc_launch_count(const Tiling &tl, int n, bool grad, long long gbuf_tiles);

// Pose vector-Jacobian product of the forward model: per-tile gradient
// moments of sum_pix r_pix sim_pix into gpart (contracted per patch by
// launch_ncc_finish with part = null).
cudaError_t launch_pose_vjp(const PsfTab &psf, const Tiling &tl, int nx, int ny, int nz,
                            const float *x, const float *r, const int32_t *desc,
                            const int32_t *fix, int n, double *gpart, float *gbuf,
                            long long gbuf_tiles, int *counter, cudaStream_t st);

// part == null: only the gradient (from gpart), no NCC.  poses and grad:
// float64 [n][n_params].
cudaError_t launch_ncc_finish(const DevGeom *g, const int32_t *desc, const double *poses, int n_params,
                              int n, const Tiling &tl, const double *part, const double *gpart,
                              int min_valid, double *ncc, double *grad, cudaStream_t st);

// Registration state: best / gbest [n][kRegStride], trial and grad [n][n_params].
cudaError_t launch_reg_init(const double *poses, int n_params, int n, double *best, double *trial,
                            double *delta, int32_t *active, double delta0, cudaStream_t st);

cudaError_t launch_reg_step(const DevGeom *g, const int32_t *desc, int n, int eval, int last,
                            const double *ncc, const double *grad, double *best, double *gbest,
                            double *nbest, double *trial, double *delta, int32_t *active,
                            const pvr_params &prm, cudaStream_t st);

cudaError_t launch_reg_finish(const double *best, const double *nbest, int n_params, int n, double *poses,
                              double *ncc_out, cudaStream_t st);


cudaError_t launch_patches_gather(const DevGeom *g, const float *stacks, const int32_t *desc,
                                  int n, int64_t n_pix, int32_t *err, float *y, cudaStream_t st);

cudaError_t launch_patch_metrics(const float *y, const float *sim, const uint8_t *valid, const int32_t *desc,
                                 int n, int w, int max_side, double *out, float *map, cudaStream_t st);

cudaError_t launch_metrics(const float *ref, const float *img, const uint8_t *mask, int64_t n,
                           double *scratch, double *out, cudaStream_t st);

}  // namespace pvr
