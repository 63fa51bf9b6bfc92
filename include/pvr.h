/*
 * pvr.h -- C ABI of the B300 (sm_103a) PVR hot-path library, libpvr.so.
 *
 * PVR (patch-to-volume reconstruction, Alansary et al., arXiv:1611.07289)
 * reconstructs a high-resolution volume x from many small 2-D patches y_s of
 * motion-corrupted slice stacks (Sec. II, Eq. patch), each patch with its own
 * rigid or affine pose, by alternating patch-to-volume registration with NCC (Sec. II),
 * super-resolution through the PSF forward model x_i = W_i y + n_i,
 * W_i = D B T_i (Eq. 1) and its adjoint, and EM outlier rejection at pixel
 * and patch level (Sec. II, Eqs. m, p, p-bar).
 *
 * Conventions (all entry points):
 *  - Every array argument is a DEVICE pointer owned by the caller, unless the
 *    argument is documented as host.  The library never frees or keeps them.
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL = the legacy default stream), except where "synchronises" is
 *    stated.  No call allocates memory: the scratch a call needs was
 *    allocated by pvr_ctx_create, sized by pvr_params.max_patches /
 *    max_pixels.
 *  - Return value: PVR_OK (0) or a negative pvr_status.  Arguments are
 *    checked on the host before anything is launched; on error nothing is
 *    enqueued and pvr_last_error(ctx) gives a one-line message.  Problems
 *    only the device can see (a patch row outside its stack, a non-finite
 *    pose) set a device error word instead: the offending patch is treated
 *    as empty and pvr_device_status() reports the error later.
 *  - Layouts: volume [nz][ny][nx] float32, x fastest.  Stacks: one packed
 *    float32 buffer, stack after stack, each [K][H][W].  Patch table:
 *    int32 [n][8] rows {stack, slice, x0, y0, w, h, pix_off, 0}: the patch
 *    covers columns x0..x0+w-1, rows y0..y0+h-1 of the slice; its pixels are
 *    stored row-major at pix_off .. pix_off + w*h - 1 of every per-pixel
 *    array.  Poses: float64 [n][n_params] (pvr_params.n_params).
 *    Rigid (6): (tx, ty, tz in mm, rx, ry, rz in degrees), transform
 *    T(w) = R (w - c) + c + t, R = Rz Ry Rx.  Affine (12): (tx, ty, tz in
 *    mm, d00, d01, d02, d10, ..., d22), T(w) = (I + D)(w - c) + c + t with D
 *    the 3x3 matrix given row-major (Eq. 1: T_i is the patch's motion; Sec.
 *    II registers patches under rigid or affine motion).  c = world centre
 *    of the patch rectangle; T maps an acquired sample position (scanner
 *    world) to the reconstruction's world frame.  Pose gradients have the
 *    same [n][n_params] layout.
 *  - Geometry: 3x4 row-major affine matrices (implied last row 0 0 0 1):
 *    world_to_voxel maps mm to voxel index (voxel centres at integers);
 *    pixel_to_world[s] maps (column, row, slice) of stack s to mm.
 *
 * Thread safety: one pvr_ctx may be used from one host thread at a time;
 * calls on one context that overlap on the GPU (different streams) race on
 * its scratch.  Separate contexts are independent.
 */
#ifndef PVR_H
#define PVR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PVR_API __attribute__((visibility("default")))
#else
#define PVR_API
#endif

#define PVR_MAX_STACKS 16
#define PVR_MAX_KXY 3
#define PVR_MAX_KZ 8
#define PVR_PSF_GAUSSIAN 0
#define PVR_PSF_TAYLOR_SINC 1
#define PVR_EM_STATE_LEN 16

typedef enum pvr_status {
    PVR_OK = 0,
    PVR_ERR_INVALID_ARG = -1, /* bad argument or capacity exceeded (host check) */
    PVR_ERR_CUDA = -2,        /* a CUDA runtime call failed */
    PVR_ERR_NUMERIC = -3,     /* non-finite pose or state seen on the device */
    PVR_ERR_BOUNDS = -4,      /* a patch row outside its stack / pixel range */
    PVR_ERR_TIMEOUT = -5,     /* a bounded device wait gave up */
    PVR_ERR_UNSUPPORTED = -6  /* valid request this build does not implement */
} pvr_status;

/* EM state vector (float64, device, PVR_EM_STATE_LEN entries).  Zero it
 * before the first pvr_em_weights / pvr_reconstruct_iter call. */
enum pvr_em_state_index {
    PVR_ST_INIT = 0,      /* 0 until the first EM call has initialised it */
    PVR_ST_SIGMA2 = 1,    /* inlier residual variance sigma^2 (Sec. II) */
    PVR_ST_C = 2,         /* inlier proportion c */
    PVR_ST_M = 3,         /* outlier density m = 1/(max e - min e) of the last call */
    PVR_ST_MU_P = 4,      /* patch-level inlier mean of p-bar */
    PVR_ST_SIGMA2_P = 5,  /* patch-level inlier variance */
    PVR_ST_C_P = 6,       /* patch-level inlier proportion */
    PVR_ST_M_P = 7,       /* patch-level outlier density */
    PVR_ST_N_PART = 8,    /* participating pixels of the last call */
    PVR_ST_SUM_P = 9,     /* sum p over them */
    PVR_ST_SUM_PE2 = 10,  /* sum p e^2 over them */
    PVR_ST_EMIN = 11,     /* min e */
    PVR_ST_EMAX = 12,     /* max e */
    PVR_ST_N_ELIG = 13,   /* patches eligible for classification */
    PVR_ST_N_IN = 14,     /* patches classified inlier */
    PVR_ST_SIGMA2_USED = 15 /* sigma^2 used by the E-step of the last call */
};

typedef struct pvr_geometry {
    int32_t nx, ny, nz;                             /* volume size, each 2..2048, nx*ny*nz < 2^31 */
    int32_t n_stacks;                               /* 1..PVR_MAX_STACKS */
    int32_t stack_w[PVR_MAX_STACKS];                /* columns */
    int32_t stack_h[PVR_MAX_STACKS];                /* rows */
    int32_t stack_k[PVR_MAX_STACKS];                /* slices */
    double world_to_voxel[12];                      /* 3x4, mm -> voxel index */
    double pixel_to_world[PVR_MAX_STACKS][12];      /* 3x4, (col,row,slice) -> mm */
    double thickness[PVR_MAX_STACKS];               /* slice thickness = through-plane FWHM, mm */
} pvr_geometry;

typedef struct pvr_params {
    /* Gaussian PSF (Sec. II; the Gaussian approximation of the cited prior
     * work).  In-plane taps at pixel offsets -kxy..kxy with weight
     * exp(-d^2 / 2 sigma_xy^2), sigma_xy = fwhm_xy / (2 sqrt(2 ln 2)) px;
     * through-plane samples at zeta * dz mm, zeta = -kz..kz, weight
     * exp(-(zeta dz)^2 / 2 sigma_z^2), sigma_z = thickness / (2 sqrt(2 ln 2)). */
    double psf_fwhm_xy;     /* pixels (default 1.2) */
    int32_t psf_kxy;        /* 0..PVR_MAX_KXY (default 1) */
    int32_t psf_kz;         /* 0..PVR_MAX_KZ (default 3) */
    double psf_dz;          /* mm, > 0 (default 1.0; use the voxel size) */
    /* super-resolution (weighted SIRT) */
    double alpha;           /* step, 0 < alpha < 2 (default 1) */
    double conf_eps;        /* voxels with A^T w <= conf_eps are not updated (1e-6) */
    /* EM outlier model */
    double em_c0;           /* initial inlier proportion (0.9) */
    double em_sigma_floor_rel; /* sigma^2 >= (rel * range e)^2 (1e-3) */
    double em_min_valid_frac;  /* patches with fewer valid pixels are excluded (0.1) */
    int32_t patch_rule;     /* 0: Gaussian/uniform patch model, 1: threshold */
    double patch_threshold; /* rule 1 threshold on p-bar (0.5) */
    int32_t patch_em_iters; /* patch-level EM iterations per call (5) */
    /* registration */
    int32_t n_params;       /* 6 = rigid, 12 = affine (pose layout above) */
    int32_t reg_evals;      /* NCC evaluations per registration round (40) */
    double reg_delta0;      /* initial step in scaled units (2) */
    double reg_delta_min;   /* stop below this step (0.01) */
    double reg_grow;        /* step factor after an accepted trial (1) */
    int32_t reg_fixed_step; /* 1: always accept, constant step */
    int32_t reg_min_valid;  /* fewer valid pixels: NCC = 0, no update (16) */
    /* outer iteration */
    int32_t n_sr;           /* SR passes per pvr_reconstruct_iter (1) */
    /* capacity of the context's scratch */
    int32_t max_patches;    /* largest patch count of any call */
    int64_t max_pixels;     /* largest total pixel count of any call */
    int32_t max_patch_side; /* largest patch width or height (1..256) */
    /* in-plane PSF profile: PVR_PSF_GAUSSIAN (above) or PVR_PSF_TAYLOR_SINC:
     * weight sinc(1.2067091288 d / psf_fwhm_xy), sinc(u) = sin(pi u)/(pi u)
     * (full width at half maximum psf_fwhm_xy pixels) summed from its Taylor
     * series until a term is below psf_sinc_eps times the sum (Sec. II); the
     * slice profile stays Gaussian.  Weights may be negative; a pixel whose
     * PSF weight sum is not positive is invalid. */
    int32_t psf_kind;       /* default PVR_PSF_GAUSSIAN */
    double psf_sinc_eps;    /* default 1e-12 */
    /* superpixel patch builder: the smallest superpixel size a the context
     * serves (its scratch is sized for it at creation); 0 (default): no
     * superpixel scratch, pvr_patches_build_slic is refused */
    int32_t slic_a_min;
    /* regularised super-resolution update: after the SIRT step every voxel
     * the data reached takes one edge-preserving diffusion step over its 26
     * neighbours, x += sr_lambda * sum_d w_d psi(x_d - x), psi(D) =
     * D / sqrt(1 + (D / sr_edge_delta)^2), w_d = (1/|d|^2) / (44/3) (the
     * anisotropic-diffusion regularisation of the SR framework PVR follows,
     * Sec. I and II), then x = max(x, 0).  sr_lambda 0 (default): plain
     * SIRT; 0..1.  sr_edge_delta > 0, intensity units (default 100). */
    double sr_lambda;
    double sr_edge_delta;
} pvr_params;

/* Patch table handed to every per-patch call (host struct, device table). */
typedef struct pvr_patches {
    const int32_t *desc;    /* device int32 [n][8], see layout above */
    int32_t n;              /* number of patches, 0..max_patches */
    int32_t max_side;       /* largest w or h in the table (0: max_patch_side) */
    int64_t n_pix;          /* pixels: every pix_off + w*h <= n_pix <= max_pixels */
    const uint8_t *member;  /* device uint8 [n_pix] or NULL: pixels with member 0 lie in
                               their patch's rectangle but not in the patch (superpixel
                               patches); they are invalid everywhere */
} pvr_patches;

typedef struct pvr_ctx pvr_ctx;

/* Fill *p with the defaults listed above (max_patches 65536,
 * max_pixels 2^27, max_patch_side 128). */
PVR_API void pvr_params_default(pvr_params *p);

/* Create a context on the current CUDA device: copies the geometry and the
 * parameters, derives the PSF tables and allocates all scratch (the only
 * allocation the library makes).  Synchronises.  Errors:
 * PVR_ERR_INVALID_ARG for a bad geometry/parameter, PVR_ERR_CUDA when an
 * allocation fails (*out is then NULL). */
PVR_API int pvr_ctx_create(pvr_ctx **out, const pvr_geometry *geom, const pvr_params *params);

/* Free the context and its scratch (synchronises the device).  NULL is a no-op. */
PVR_API int pvr_ctx_destroy(pvr_ctx *ctx);

/* Last host-side error message of this context ("" if none). */
PVR_API const char *pvr_last_error(const pvr_ctx *ctx);

/* Synchronise `stream`, read and clear the device error word: PVR_OK,
 * PVR_ERR_BOUNDS, PVR_ERR_NUMERIC or PVR_ERR_TIMEOUT (a bounded device wait
 * gave up; the affected output is not valid). */
PVR_API int pvr_device_status(pvr_ctx *ctx, void *stream);

/* Number of kernel launches this context has enqueued since creation
 * (host counter; for launch accounting). */
PVR_API int64_t pvr_launch_count(const pvr_ctx *ctx);

/* Kernel classes of the optional launch profiler. */
enum pvr_kernel_class {
    PVR_K_POSE = 0,      /* pose -> fixed-point lattice */
    PVR_K_SIMULATE = 1,  /* forward model (+ residual) */
    PVR_K_EM = 2,        /* EM statistics, E-step, M-step + patch classification */
    PVR_K_ADJOINT = 3,   /* adjoint scatter */
    PVR_K_UPDATE = 4,    /* SIRT volume update */
    PVR_K_NCC = 5,       /* NCC moments + pose gradient */
    PVR_K_NCC_FINISH = 6,/* per-patch NCC / gradient fold */
    PVR_K_REG_STEP = 7,  /* registration accept / propose */
    PVR_K_N = 8
};

/* Optional launch profiler (measurement aid, not part of the method).
 * enable = 1: from now on every launch of the classes above made by this
 * context is bracketed by CUDA events recorded on the launch's own stream
 * (an event pool of fixed size is created on the first enable; when it runs
 * out, further launches are not recorded).  enable = 0 stops recording. */
PVR_API int pvr_profile_enable(pvr_ctx *ctx, int32_t enable);

/* Synchronise `stream`, then write per class the summed device time (ms,
 * HOST array [PVR_K_N]) and the number of recorded launch groups (HOST
 * array [PVR_K_N], may be NULL) since the last read, and reset. */
PVR_API int pvr_profile_read(pvr_ctx *ctx, double *ms, int64_t *launches, void *stream);

/* Square patch table (Sec. II "Patch Extraction": size a, stride `stride`).
 * Candidates x0, y0 = 0, stride, 2 stride, ... with x0 + a <= W, y0 + a <= H,
 * on every slice of every stack, ordered by stack, slice, y0, x0.  A
 * candidate is kept when at least keep_frac * a^2 of its pixels exceed
 * fg_frac * I_max (I_max = largest stack pixel; level and comparisons in
 * float32, count test in float64).  stacks: device float32, packed.
 * desc_out: device int32 [max_out][8].  n_out, n_pix_out: HOST pointers;
 * the call synchronises `stream` to return them.  If more than max_out
 * patches are kept, *n_out is the full count and only max_out rows are
 * written.  The fixed-point lattice and every later step take the table as
 * is, so caller-made tables (uneven patch sizes) are equally valid. */
PVR_API int pvr_patches_build(pvr_ctx *ctx, const float *stacks, int32_t a, int32_t stride,
                      double fg_frac, double keep_frac, int32_t *desc_out, int32_t max_out,
                      int32_t *n_out, int64_t *n_pix_out, void *stream);

/* The same with a side and stride per slice: slice_a, slice_stride are HOST
 * int32 arrays with one entry per slice of every stack, numbered over the
 * stacks in order (multi-scale patch sets: Sec. II extracts patches at
 * several sizes).  Candidates of a slice use that slice's side and stride;
 * pixel offsets are packed over the kept patches in table order.  Each side
 * must be 1..max_patch_side and each stride >= 1; the total candidate pixel
 * count must stay below 2^31. */
PVR_API int pvr_patches_build_sizes(pvr_ctx *ctx, const float *stacks, const int32_t *slice_a,
                                    const int32_t *slice_stride, double fg_frac, double keep_frac,
                                    int32_t *desc_out, int32_t max_out, int32_t *n_out,
                                    int64_t *n_pix_out, void *stream);

/* Superpixel patch table (Sec. II "Patch Extraction": SLIC superpixels of
 * initial size a and compactness t, D^2 = d_c^2 + (d_s / a)^2 t^2, dilated by
 * gamma pixels with a square element).  Every superpixel of every slice
 * whose dilated bounding box fits min(max_patch_side, 128) becomes a row
 * {stack, slice, x0, y0, w, h, pix_off, 0} (box of the dilated superpixel)
 * when at least keep_frac of its member pixels exceed fg_frac * I_max;
 * member_out (device uint8, capacity max_pixels) receives, per box pixel,
 * 1 if it belongs to the dilated superpixel: pass it as pvr_patches.member.
 * Centres start on a grid of max(1, round(W/a)) x max(1, round(H/a)) cells;
 * n_iter assignment/update rounds (integer intensity sums, so the result
 * does not depend on the summation order).  a >= pvr_params.slic_a_min
 * (>= 2); gamma 0..32; n_iter 1..100.  Uses the context's superpixel scratch
 * (allocates nothing); synchronises `stream`; n_out, n_pix_out: HOST
 * pointers. */
PVR_API int pvr_patches_build_slic(pvr_ctx *ctx, const float *stacks, int32_t a, double compactness,
                                   int32_t gamma, int32_t n_iter, double fg_frac, double keep_frac,
                                   int32_t *desc_out, uint8_t *member_out, int32_t max_out,
                                   int32_t *n_out, int64_t *n_pix_out, void *stream);

/* Copy every patch's pixels out of the packed stacks into y (float32
 * [n_pix], patch after patch, row-major). */
PVR_API int pvr_patches_gather(pvr_ctx *ctx, const float *stacks, const pvr_patches *patches, float *y,
                       void *stream);

/* Pose -> fixed-point sample lattice (Eq. 1, the motion part T_i of W_i).
 * For each patch, M = world_to_voxel . T(theta) . pixel_to_world[stack]
 * evaluated in float64 with a fixed operation order (no FMA; sine and
 * cosine from their Taylor series after reduction to +-45 degrees), then
 * quantised to Q11.20 (round half to even): fix int32 [n][16] =
 * {o(3), e_col(3), e_row(3), e_zeta(3), ok, 0, 0, 0}; o = voxel position of
 * patch pixel (0,0), e_col / e_row = one pixel step, e_zeta = one PSF step
 * of psf_dz mm along the slice normal.  ok = 0 when the patch's sample box
 * leaves +-1024 voxels or a value does not fit (the patch is then empty). */
PVR_API int pvr_pose_to_fixed(pvr_ctx *ctx, const pvr_patches *patches, const double *poses,
                      int32_t *fix, void *stream);

/* Forward model simulate_patches (Eq. 1; Sec. II super-resolution): every
 * patch pixel is the PSF-weighted mean of trilinear samples of x at its
 * transformed sample positions (samples outside the volume carry no
 * weight).  sim: float32 [n_pix]; valid: uint8 [n_pix], 0 where no sample
 * fell inside (sim = 0 there). */
PVR_API int pvr_simulate(pvr_ctx *ctx, const float *x, const pvr_patches *patches, const double *poses,
                 float *sim, uint8_t *valid, void *stream);

/* pvr_simulate without a context and without any device allocation.  (The
 * paper has no counterpart: this is a deployment variant.)  For callers
 * that cannot call cudaMalloc -- e.g. a host application whose own pool
 * allocator owns the device memory and forbids other allocations, or a
 * latency-bound loop that must not allocate (allocation can synchronise the
 * device) once it is running.  Same inputs and outputs as pvr_simulate, with
 * the geometry and parameters passed per call; the scratch it needs (device
 * copy of the geometry, per-patch fixed-point table, error word) lives in a
 * fixed device array inside the library that every GPU loading the library
 * keeps until the process exits.  Limits: patches->n <= 8192 (more:
 * PVR_ERR_INVALID_ARG, nothing enqueued); n_pix < 2^31; max_side <= 256.
 * The first call on a device looks the array up with that device current;
 * make that first call before any stream capture begins.  All calls share
 * the one array: calls that overlap on the GPU race, so serialise them.
 * The geometry and the PSF / pose settings pass the checks of
 * pvr_ctx_create (PVR_ERR_INVALID_ARG, nothing enqueued); n_params 6 or 12.
 * A malformed patch row is skipped (its pixels are not written) and a pose
 * whose sample map is not finite leaves its patch without valid pixels;
 * both set the array's error word, which pvr_noalloc_status reports (there
 * is no context, so no error message). */
PVR_API int pvr_simulate_noalloc(const pvr_geometry *geom, const pvr_params *params, const float *x,
                                 const pvr_patches *patches, const double *poses, float *sim,
                                 uint8_t *valid, void *stream);

/* Error word of pvr_simulate_noalloc on the current device: synchronises
 * `stream`, reads the word and clears it.  It collects every call since the
 * last read: PVR_OK, PVR_ERR_BOUNDS (a patch row outside its stack or
 * pixel range) or PVR_ERR_NUMERIC (a pose with a non-finite sample map).
 * Allocates nothing; the same sharing rule as pvr_simulate_noalloc applies.
 * (The paper has no counterpart: part of the deployment variant.) */
PVR_API int pvr_noalloc_status(void *stream);

/* Adjoint of pvr_simulate (the super-resolution update's back-projection):
 * addon = A^T (w .* r), conf = A^T w, A the matrix of pvr_simulate at these
 * poses.  r, w: float32 [n_pix] or NULL (= all ones).  addon, conf: float32
 * [nx*ny*nz], either may be NULL (skipped).  accumulate = 0 zeroes them
 * first, 1 adds.  Summation order on the device is not fixed (float atomics). */
PVR_API int pvr_adjoint(pvr_ctx *ctx, const pvr_patches *patches, const double *poses, const float *r,
                const float *w, float *addon, float *conf, int32_t accumulate, void *stream);

/* EM outlier weights (Sec. II "EM-Based Outlier Removal", Eqs. m, p, p-bar).
 * e = y - sim on valid pixels (sim == NULL: y already holds e).
 * Participating pixels = valid pixels of patches with mask_in = 1
 * (mask_in == NULL: all).  First call (state[INIT] == 0): sigma^2 = mean e^2,
 * c = em_c0.  m = 1/(max e - min e) over participating pixels (0 if the range
 * is < 1e-12).  E-step on every valid pixel: p = G c / (G c + m (1 - c)),
 * G = N(e; 0, sigma^2), p = 1 if m = 0, p = 0 on invalid pixels.  M-step
 * over participating pixels: sigma^2 = sum p e^2 / sum p (floored), c =
 * sum p / N.  Patch potential p-bar = sqrt(sum p^2 / N_valid) per patch;
 * patches with N_valid < em_min_valid_frac * w * h are excluded; the rest are
 * classified by patch_rule (0: one-sided Gaussian inlier vs uniform outlier
 * model on p-bar, patch_em_iters EM iterations, w_patch = inlier posterior,
 * mask = w_patch >= 0.5; 1: w_patch = p-bar, mask = p-bar >= threshold).
 * state: float64 device [PVR_EM_STATE_LEN], in/out.  p: float32 [n_pix];
 * w_patch, pbar: float32 [n] (pbar may be NULL); mask_out: uint8 [n]
 * (must not alias mask_in). */
PVR_API int pvr_em_weights(pvr_ctx *ctx, const float *y, const float *sim, const uint8_t *valid,
                   const pvr_patches *patches, double *state, const uint8_t *mask_in,
                   uint8_t *mask_out, float *p, float *w_patch, float *pbar, void *stream);

/* Weighted SIRT step of the super-resolution update (rows of A sum to one):
 * where conf > conf_eps, x = max(x + alpha * addon / conf, 0); with
 * sr_lambda > 0 followed by the edge-preserving diffusion step on those
 * voxels (pvr_params).  If clear_accumulators, addon and conf are zeroed. */
PVR_API int pvr_volume_update(pvr_ctx *ctx, float *x, float *addon, float *conf, int32_t clear_accumulators,
                      void *stream);

/* Initial volume x = A^T y / A^T 1 (0 where A^T 1 <= conf_eps) at `poses`. */
PVR_API int pvr_volume_init(pvr_ctx *ctx, float *x, const float *y, const pvr_patches *patches,
                    const double *poses, void *stream);

/* Per-patch evaluation against the acquired patches (Sec. IV-A: metrics
 * between original 2D patches and patches simulated from the
 * reconstruction).  Over each patch's valid pixels, with the acquired patch
 * y as reference: out[5p..5p+4] = {PSNR = 10 log10(I_max^2 / MSE), CC,
 * SSIM (global, c1 = (0.01 L)^2, c2 = (0.03 L)^2, L = range of y), DSSIM =
 * (1 - SSIM)/2, mean local SSIM}; map (may be NULL): the DSSIM heat map,
 * per valid pixel (1 - SSIM)/2 over the valid pixels of its (2w+1)^2
 * window clipped to the patch, 0 at invalid pixels.  out: float64 [n][5];
 * map: float32 [n_pix]; w: 0..16. */
PVR_API int pvr_patch_metrics(pvr_ctx *ctx, const float *y, const float *sim, const uint8_t *valid,
                              const pvr_patches *patches, int32_t w, double *out, float *map,
                              void *stream);

/* Rigidity (data-consistency) map (Sec. II, "Identification of Rigid
 * Regions"): the pixel probabilities p and patch potentials p-bar
 * integrated into the volume with the reconstruction's PSF,
 * out = A^T(p * pbar_patch) / A^T 1 where A^T 1 > conf_eps, else 0 -- the
 * PSF-weighted mean of p * p-bar over the samples that reach each voxel.
 * p: float32 [n_pix] (e.g. pvr_em_weights' p); pbar: float32 [n] (p-bar or
 * the patch weight); out: float32 volume. */
PVR_API int pvr_rigidity_map(pvr_ctx *ctx, const pvr_patches *patches, const double *poses,
                             const float *p, const float *pbar, float *out, void *stream);

/* NCC of every patch against the volume simulated at its pose, and its
 * gradient with respect to the n_params pose parameters (Sec. II: CC similarity,
 * Eq. cross_corr with population deviations, over valid pixels; the PSF
 * normalisation is held constant in the derivative).  Fewer than
 * reg_min_valid valid pixels or a constant patch: NCC = 0, gradient 0.
 * ncc: float64 [n]; grad: float64 [n][n_params] (may be NULL). */
PVR_API int pvr_ncc_grad(pvr_ctx *ctx, const float *x, const float *y, const pvr_patches *patches,
                 const double *poses, double *ncc, double *grad, void *stream);

/* Pose gradient of sum_pix r_pix sim_pix for every patch: the
 * vector-Jacobian product of pvr_simulate with respect to the poses, the
 * backward pass of a differentiable forward model (Eq. 1 differentiated
 * through the sample positions; the PSF normalisation is held constant, as
 * in pvr_ncc_grad).  Together with pvr_adjoint (the product with respect to
 * x) it gives both gradients of any loss of the simulated patches.  The PSF
 * weights are recomputed, nothing is stored by the forward call.
 * x: float32 volume; r: float32 [n_pix] (dL/dsim; invalid pixels ignored);
 * poses, grad (out): float64 [n][n_params].  This entry point extends
 * the paper's method (the paper differentiates only NCC). */
PVR_API int pvr_pose_grad(pvr_ctx *ctx, const float *x, const float *r, const pvr_patches *patches,
                          const double *poses, double *grad, void *stream);

/* Patch-wise gradient ascent on NCC (Sec. II; Sec. III "patch-wise gradient
 * descent"): n_evals NCC evaluations per patch, the first at the current
 * pose, then trials best + delta * g/|g| in scaled units (translations in
 * mm, rigid angles x patch half-diagonal in radians, affine entries x patch
 * half-diagonal: one unit moves the patch edge by about 1 mm); a trial that
 * strictly improves NCC is kept (delta *= reg_grow), otherwise delta halves;
 * a patch stops when delta < reg_delta_min.  reg_fixed_step: always accept.
 * poses: float64 [n][n_params] in/out; ncc: float64 [n] best NCC (may be
 * NULL). */
PVR_API int pvr_register(pvr_ctx *ctx, const float *x, const float *y, const pvr_patches *patches,
                 double *poses, int32_t n_evals, double *ncc, void *stream);

/* One outer PVR iteration (Sec. II loop): pvr_register with reg_evals
 * evaluations, then n_sr super-resolution passes, each: simulate, residual
 * e = y - sim, EM weights (mask carried from pass to pass), weighted adjoint
 * of e with pixel weight mask_patch * p, SIRT update of x (with the
 * edge-preserving diffusion step when sr_lambda > 0).  x: in/out;
 * poses: in/out; state: EM state in/out; mask: uint8 [n] in/out (set to 1
 * before the first call); p (float32 [n_pix]) and w_patch (float32 [n])
 * receive the last pass's weights (either may be NULL).  When every patch
 * is one tile (sides <= 64 pixels and no 32-pixel launch plan), the
 * registration's NCC evaluations already compute the forward model at each
 * patch's best pose; the first pass uses it instead of simulating again
 * (the same values up to float32 summation order). */
PVR_API int pvr_reconstruct_iter(pvr_ctx *ctx, float *x, const float *y, const pvr_patches *patches,
                         double *poses, double *state, uint8_t *mask, float *p, float *w_patch,
                         void *stream);

/* Work plan for one patch table (batched patches of uneven sizes): the
 * table's non-empty (patch, tile) slots ordered largest tile first, served by
 * persistent simulate / adjoint kernels that take tiles from an atomic work
 * queue (mode 1), or one CTA per slot (mode 0), with tile side 64 or 32.
 * tile: 0 = tune, 32 or 64; mode: -1 = tune, 0 or 1.  Tuning times each
 * candidate (simulate with residual + adjoint, 3 runs after a warm-up) on
 * x, y, poses and keeps the fastest; it synchronises `stream`.  The plan
 * applies to later pvr_simulate, pvr_adjoint and pvr_reconstruct_iter calls
 * with this same table (device pointer, n, n_pix); NCC and registration keep
 * their own tiling.  The plan also fixes a launch order of the table's
 * patches for every per-tile kernel (simulate, adjoint, NCC with and without
 * gradient, pose gradient; the work queue's items within each tile size):
 * patches sorted by the block of 32^3 voxels holding their centre at the
 * identity pose (z block, then y, then x), so that the CTAs running at one
 * time read a compact part of the volume.  Results do not depend on it
 * except for the float32 summation order of the adjoint's reductions.
 * Reads the table to the host and synchronises. */
PVR_API int pvr_plan(pvr_ctx *ctx, const pvr_patches *patches, const float *x, const float *y,
                     const double *poses, int32_t tile, int32_t mode, void *stream);

/* The current plan: tile side (0 if none), mode (-1 if none), listed tiles. */
PVR_API int pvr_plan_info(const pvr_ctx *ctx, int32_t *tile, int32_t *mode, int32_t *n_items);

/* The plan's patch launch order (a permutation of 0 .. n-1; n = the planned
 * table's patch count) copied to HOST memory host_out[n].  PVR_ERR_INVALID_ARG
 * without a plan or for another n.  Synchronises `stream`. */
PVR_API int pvr_plan_order(pvr_ctx *ctx, int32_t *host_out, int32_t n, void *stream);

/* Drop the plan (later calls use one CTA per 64-pixel tile slot). */
PVR_API int pvr_plan_clear(pvr_ctx *ctx);

/* Capture one pvr_reconstruct_iter with these arguments into a CUDA graph
 * held by the context (replacing any earlier one); nothing runs.  stream
 * must be a non-default stream; the profiler must be off.  The graph keeps
 * the pointers and the context's scratch, so replays read and write the
 * same buffers. */
PVR_API int pvr_graph_capture(pvr_ctx *ctx, float *x, const float *y, const pvr_patches *patches,
                              double *poses, double *state, uint8_t *mask, float *p, float *w_patch,
                              void *stream);

/* Replay the captured iteration on `stream`. */
PVR_API int pvr_graph_launch(pvr_ctx *ctx, void *stream);

/* ---- learned pose proposal (a small CNN; extends the paper's method) ----
 * The network reads, per 64x64 patch, the acquired pixels y and the pixels
 * simulated at the current pose s (each normalised to zero mean and unit
 * deviation over the valid pixels) and predicts the 6 rigid parameters of
 * the correction in the frame of the patch's stack: translation along and
 * rotation (degrees) about its unit column, row and slice-normal directions
 * (the frame in which the image content of any stack moves alike); six 3x3
 * bf16 convolutions (tensor cores, float32 accumulation), a float32 linear
 * head on the flattened 4x4x64 last activation.  Training is mean squared
 * error against given targets with Adam. */
typedef struct pvr_net pvr_net;

/* Allocates the network, its Adam state and activations for batches of up to
 * batch_max (1..4096) patches; weights initialised from seed. */
PVR_API int pvr_net_create(pvr_net **out, int32_t batch_max, uint64_t seed);
PVR_API int pvr_net_destroy(pvr_net *net);
/* Number of float32 parameters (conv weights [co][ky][kx][ci] and bias per
 * layer, then the head [6][1024] over the last activation in its (y, x,
 * channel) order, and its bias). */
PVR_API int64_t pvr_net_param_count(const pvr_net *net);
/* Copy the float32 parameters to / from HOST memory (set resets Adam). */
PVR_API int pvr_net_get_params(pvr_net *net, float *host_out);
PVR_API int pvr_net_set_params(pvr_net *net, const float *host_in);
/* Gradients of the last pvr_net_train_step, to HOST memory. */
PVR_API int pvr_net_get_grads(pvr_net *net, float *host_out);
/* Predictions for patches first .. first+count-1 of the table (count <=
 * batch_max; the table's max_side must be 64 and rows that are not 64x64
 * read as empty).  y, s: float32 [n_pix]; valid: uint8 [n_pix] (pixels of s
 * that are valid); out: device float32 [count][6]. */
PVR_API int pvr_net_forward(pvr_net *net, const float *y, const float *s, const uint8_t *valid,
                            const pvr_patches *patches, int32_t first, int32_t count, float *out,
                            void *stream);
/* One Adam step (learning rate lr) on the loss mean over the batch of
 * sum_j (out_j - target_j)^2; target: device float32 [count][6]; loss (device
 * float32 [1], may be NULL) receives the batch loss before the step. */
PVR_API int pvr_net_train_step(pvr_net *net, const float *y, const float *s, const uint8_t *valid,
                               const pvr_patches *patches, int32_t first, int32_t count,
                               const float *target, float lr, float *loss, void *stream);

/* Synchronise `stream`, read and clear the network's device status: PVR_OK
 * or PVR_ERR_TIMEOUT when a bounded wait of a tensor-core convolution gave
 * up since the last read (its outputs are then not valid). */
PVR_API int pvr_net_status(pvr_net *net, void *stream);

/* Scratch of pvr_pose_propose for tables of up to max_patches patches and
 * max_pixels pixels (allocates; call once before proposing). */
PVR_API int pvr_net_reserve(pvr_net *net, int32_t max_patches, int64_t max_pixels);

/* Learned pose proposal with fallback: simulate every 64x64 patch at its
 * pose, let the network predict a correction (output k times scale[k], a
 * HOST double[6], mm and degrees in the stack frame), map it to world pose
 * increments with the stack's unit axes S (translation S t, angles S w:
 * rotation about the stack axes to first order), evaluate NCC at the plain
 * and at the corrected pose, and keep the corrected pose only where NCC
 * rises.
 * The network predicts rigid corrections: the context must use rigid poses
 * (n_params 6; otherwise PVR_ERR_UNSUPPORTED).  poses: float64 [n][6]
 * in/out; accepted (device int32 [n], may be NULL):
 * 1 where the proposal was taken.  Run NCC registration (pvr_register /
 * pvr_reconstruct_iter) afterwards to refine. */
PVR_API int pvr_pose_propose(pvr_ctx *ctx, pvr_net *net, const float *x, const float *y,
                             const pvr_patches *patches, const double *scale, double *poses,
                             int32_t *accepted, void *stream);

/* Evaluation metrics (Sec. IV-A) of img against ref over n values (mask
 * NULL: all): out float64 device [5] = {PSNR = 10 log10(I_max^2/MSE),
 * CC (Eq. cross_corr), SSIM (single global window, Eq. SSIM with the
 * denominator's first factor mu_I^2 + mu_J^2 + c1), DSSIM = (1-SSIM)/2, MSE}. */
PVR_API int pvr_metrics(pvr_ctx *ctx, const float *ref, const float *img, const uint8_t *mask, int64_t n,
                double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PVR_H */
