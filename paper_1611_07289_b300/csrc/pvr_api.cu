// C ABI of libpvr: context, argument checks, scratch, call sequencing.
// Every compute step runs in this library's kernels; the host only checks
// arguments, derives constants and enqueues launches.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "pvr_internal.h"

namespace pvr {
cudaError_t launch_em_stats(const float *y, const float *sim, const uint8_t *valid,
                            const int32_t *desc, int n, int64_t n_pix, const Tiling &tl,
                            int32_t *err, double *part, cudaStream_t st);
cudaError_t launch_em(const float *y, const float *sim, const uint8_t *valid, const int32_t *desc,
                      int n, int64_t n_pix, const Tiling &tl, int32_t *err, double *state,
                      const uint8_t *mask_in, uint8_t *mask_out, float *p, float *w_patch,
                      float *pbar_out, double *part, double *pstat, double *pbar, double *wsc,
                      uint8_t *elig, double *bpart, unsigned *counter, const pvr_params &prm, cudaStream_t st);
int em_launch_count(int n, const pvr_params &prm);
cudaError_t launch_patches_build(const DevGeom *g, const pvr_geometry &hg, const float *stacks,
                                 int64_t total, const int32_t *slice_a, const int32_t *slice_stride,
                                 double fg_frac, double keep_frac, int32_t *desc_out, int max_out,
                                 int32_t *keep, int64_t *n_cand_out, unsigned *imax_key,
                                 int32_t *counts, void *slice_scratch, cudaStream_t st);
size_t patches_slice_scratch_bytes(int n_slices);
cudaError_t launch_stack_max(const float *stacks, int64_t total, unsigned *imax_key, cudaStream_t st);
cudaError_t launch_patches_build_slic(const DevGeom *g, const pvr_geometry &hg, const float *stacks, int64_t total,
                                      int a, double t, int gamma, int n_iter, double fg_frac, double keep_frac,
                                      int max_side, int32_t *desc_out, int max_out, uint8_t *member_out,
                                      int64_t max_pix, unsigned *imax_key, int32_t *counts, int64_t *n_centres_out,
                                      void *scratch, cudaStream_t st);
size_t slic_scratch_bytes(const pvr_geometry &hg, int a_min, int64_t total);
}  // namespace pvr

using namespace pvr;

namespace {
constexpr int kMaxTile = 64;
constexpr int kMetricScratch = 2 * 8 * 296;
constexpr int kMaxSideLimit = 256;
}  // namespace

struct pvr_ctx {
    pvr_geometry geom;
    pvr_params prm;
    DevGeom hgeom;
    PsfTab psf;
    int device = 0;
    int64_t nvox = 0;
    int64_t stack_total = 0;
    int tpp_cap = 1;
    // device scratch
    DevGeom *d_geom = nullptr;
    int32_t *fix = nullptr;
    double *part = nullptr, *gpart = nullptr, *pstat = nullptr;
    double *epart = nullptr;   // EM tile partials of the forward model kept by the registration
    double *pbar = nullptr, *wsc = nullptr, *emblk = nullptr;
    unsigned *emcount = nullptr;   // arrival counter of the EM kernels' last-block folds (kept at 0)
    int *ncc_counter = nullptr;    // tile counter of the persistent NCC kernel
    uint8_t *elig = nullptr;
    int32_t *err = nullptr;
    double *best = nullptr, *gbest = nullptr, *nbest = nullptr, *trial = nullptr, *delta = nullptr;
    double *ncc_tmp = nullptr, *grad_tmp = nullptr;
    int32_t *active = nullptr;
    float *s_buf = nullptr, *e_buf = nullptr, *p_buf = nullptr;
    uint8_t *v_buf = nullptr, *valid_buf = nullptr, *mask_tmp = nullptr;
    float2 *acc2 = nullptr;   // interleaved (addon, conf) accumulator, one pair per voxel
    float4 *quad = nullptr;   // quad copy of the volume read by the gathers
    float *x_next = nullptr;  // regularised update's output volume (sr_lambda > 0)
    float *gbuf = nullptr;    // NCC gradient scratch (per-lattice-point gradient sums)
    long long gbuf_tiles = 0;
    int32_t *keep = nullptr;
    int64_t keep_cap = 0;
    unsigned *imax_key = nullptr;
    int32_t *counts = nullptr;
    void *slice_scr = nullptr;   // per-slice candidate table of the patch builder
    void *slic_scr = nullptr;    // superpixel builder scratch (pvr_params.slic_a_min > 0)
    int n_slices = 0;
    // work plan of one patch table (pvr_plan): tiling, launch mode, tile list
    int tpp_alloc = 1;            // slots per patch the partial buffers hold
    int32_t *plan_items = nullptr;
    int *plan_counter = nullptr;
    const int32_t *plan_desc = nullptr;
    int plan_n = -1;
    int64_t plan_npix = -1;
    Tiling plan_tl{};
    int plan_mode = 0;            // 0: one CTA per slot, 1: persistent work queue
    int plan_n_items = 0;
    int32_t *plan_order = nullptr;   // patch launch order of the planned table (Tiling::order)
    // captured reconstruct_iter (pvr_graph_capture)
    cudaGraphExec_t graph_exec = nullptr;
    int64_t graph_launches = 0;
    double *metric_scr = nullptr;
    std::string last_error;
    int64_t launches = 0;
    // optional launch profiler
    bool prof = false;
    std::vector<cudaEvent_t> evpool;
    std::vector<std::pair<int, int>> rec;   // (class, first event index)
    size_t ev_next = 0;
};

namespace {

int fail(pvr_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->last_error = buf;
    return code;
}

int cuda_check(pvr_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return PVR_OK;
    return fail(c, PVR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

Tiling make_tiling(int max_side, const pvr_patches *pp = nullptr)
{
    Tiling t;
    t.T = max_side <= kMaxTile ? max_side : kMaxTile;
    if (t.T < 1) t.T = 1;
    t.tiles_x = (max_side + t.T - 1) / t.T;
    t.tiles_y = t.tiles_x;
    t.tpp = t.tiles_x * t.tiles_y;
    t.member = pp ? pp->member : nullptr;
    return t;
}

Tiling make_tiling_t(int max_side, int T)
{
    Tiling t;
    t.T = max_side <= T ? max_side : T;
    if (t.T < 1) t.T = 1;
    t.tiles_x = (max_side + t.T - 1) / t.T;
    t.tiles_y = t.tiles_x;
    t.tpp = t.tiles_x * t.tiles_y;
    return t;
}

// The plan of this exact table (same device pointer, counts and side), if
// one was made: its tiling replaces tl and, in queue mode, its work queue is
// returned for the simulate / adjoint launches.
const WorkQueue *plan_for(pvr_ctx *c, const pvr_patches *pp, int max_side, Tiling *tl, WorkQueue *wq)
{
    if (c->plan_n < 0 || pp->desc != c->plan_desc || pp->n != c->plan_n || pp->n_pix != c->plan_npix ||
        max_side > c->plan_tl.T * c->plan_tl.tiles_x)
        return nullptr;
    *tl = c->plan_tl;
    tl->member = pp->member;
    tl->order = c->plan_order;
    if (c->plan_mode != 1) return nullptr;
    wq->items = c->plan_items;
    wq->n_items = c->plan_n_items;
    wq->counter = c->plan_counter;
    return wq;
}

// The default tiling of a table, with the planned launch order when pvr_plan
// was called on this exact table.
Tiling tiling_for(const pvr_ctx *c, int max_side, const pvr_patches *pp)
{
    Tiling t = make_tiling(max_side, pp);
    if (c->plan_n >= 0 && pp->desc == c->plan_desc && pp->n == c->plan_n && pp->n_pix == c->plan_npix)
        t.order = c->plan_order;
    return t;
}

int check_patches(pvr_ctx *c, const pvr_patches *pp, int *max_side)
{
    if (!pp) return fail(c, PVR_ERR_INVALID_ARG, "patches is NULL");
    if (pp->n < 0 || pp->n > c->prm.max_patches)
        return fail(c, PVR_ERR_INVALID_ARG, "patch count %d outside 0..%d", pp->n, c->prm.max_patches);
    if (pp->n > 0 && !pp->desc) return fail(c, PVR_ERR_INVALID_ARG, "patch table is NULL");
    if (pp->n_pix < 0 || pp->n_pix > c->prm.max_pixels)
        return fail(c, PVR_ERR_INVALID_ARG, "pixel count %lld outside 0..%lld", (long long)pp->n_pix,
                    (long long)c->prm.max_pixels);
    int ms = pp->max_side > 0 ? pp->max_side : c->prm.max_patch_side;
    if (ms > c->prm.max_patch_side)
        return fail(c, PVR_ERR_INVALID_ARG, "max_side %d above the context's %d", ms,
                    c->prm.max_patch_side);
    *max_side = ms;
    return PVR_OK;
}

#define REQUIRE(cond, ...)                                          \
    do {                                                            \
        if (!(cond)) return fail(c, PVR_ERR_INVALID_ARG, __VA_ARGS__); \
    } while (0)

#define CUDA_TRY(expr, what)                                  \
    do {                                                      \
        int _rc = cuda_check(c, (expr), what);                \
        if (_rc != PVR_OK) return _rc;                        \
    } while (0)

constexpr size_t kProfEvents = 8192;

int prof_begin(pvr_ctx *c, int cls, cudaStream_t st)
{
    if (!c->prof || c->ev_next + 2 > c->evpool.size()) return -1;
    int i = (int)c->ev_next;
    c->ev_next += 2;
    cudaEventRecord(c->evpool[i], st);
    c->rec.push_back({cls, i});
    return i;
}

void prof_end(pvr_ctx *c, int i, cudaStream_t st)
{
    if (i >= 0) cudaEventRecord(c->evpool[i + 1], st);
}

// CUDA_TRY with the launch bracketed by profiler events (when enabled).
#define CUDA_TRY_T(cls, expr, what)               \
    do {                                          \
        int _pi = prof_begin(c, (cls), st);       \
        CUDA_TRY(expr, what);                     \
        prof_end(c, _pi, st);                     \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t n)
{
    return cudaMalloc((void **)p, (n > 0 ? n : 1) * sizeof(T));
}

void free_all(pvr_ctx *c)
{
    void *ptrs[] = {c->d_geom, c->fix, c->part, c->epart, c->gpart, c->pstat, c->pbar, c->wsc, c->emblk, c->emcount, c->ncc_counter, c->elig,
                    c->err, c->best, c->gbest, c->nbest, c->trial, c->delta, c->ncc_tmp,
                    c->grad_tmp, c->active, c->s_buf, c->e_buf, c->p_buf, c->v_buf,
                    c->valid_buf, c->mask_tmp, c->acc2, c->quad, c->x_next, c->gbuf, c->keep, c->imax_key,
                    c->slice_scr, c->slic_scr, c->plan_items, c->plan_counter, c->plan_order,
                    c->counts, c->metric_scr};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
}

// Quad copy of x for the gathers (once per call that gathers from x).
int build_quad(pvr_ctx *c, const float *x, cudaStream_t st)
{
    CUDA_TRY(launch_build_quad(x, c->quad, c->geom.nx, c->geom.ny, c->geom.nz, st), "quad");
    c->launches += 1;
    return PVR_OK;
}

// K1 for a patch table at `poses` into the context's fixed table.
int pose_fixed(pvr_ctx *c, const pvr_patches *pp, int max_side, const double *poses, cudaStream_t st)
{
    CUDA_TRY_T(PVR_K_POSE, launch_pose_to_fixed(c->d_geom, pp->desc, poses, c->prm.n_params, pp->n, pp->n_pix,
                                                max_side, c->psf.kxy, c->psf.kz, c->fix, c->err, st),
             "pose_to_fixed");
    c->launches += pp->n > 0;
    return PVR_OK;
}

// The super-resolution update of x from the interleaved accumulator: the
// SIRT step, and with sr_lambda > 0 the edge-preserving diffusion step
// (into x_next, copied back); the accumulator ends cleared.  Returns the
// number of kernels launched through *launched.
int sr_update_pairs(pvr_ctx *c, float *x, cudaStream_t st, int *launched)
{
    const float alpha = (float)c->prm.alpha, eps = (float)c->prm.conf_eps;
    if (c->prm.sr_lambda <= 0.0) {
        CUDA_TRY_T(PVR_K_UPDATE, launch_volume_update_pairs(x, c->acc2, c->nvox, alpha, eps, 1, 0, st), "volume_update");
        *launched = 1;
        return PVR_OK;
    }
    CUDA_TRY_T(PVR_K_UPDATE, launch_volume_update_pairs(x, c->acc2, c->nvox, alpha, eps, 0, 0, st), "volume_update");
    CUDA_TRY_T(PVR_K_UPDATE, launch_sr_diffuse_pairs(x, c->acc2, c->x_next, c->geom.nx, c->geom.ny, c->geom.nz,
                                                     (float)c->prm.sr_lambda, (float)c->prm.sr_edge_delta, eps,
                                                     c->err, st),
               "sr_diffuse");
    CUDA_TRY(cudaMemcpyAsync(x, c->x_next, (size_t)c->nvox * sizeof(float), cudaMemcpyDeviceToDevice, st),
             "copy regularised volume");
    *launched = 2;
    return PVR_OK;
}

}  // namespace

namespace pvr {

// sin(pi u) / (pi u) summed from its Maclaurin series (Sec. II, the
// Taylor-series PSF) until a term is below eps times the sum.
double sinc_series(double u, double eps)
{
    const double x = 3.14159265358979323846 * u, x2 = x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 200; ++k) {
        term = -term * x2 / ((double)(2 * k) * (double)(2 * k + 1));
        sum += term;
        if (fabs(term) <= eps * fabs(sum)) break;
    }
    return sum;
}

void make_psf_tab(const pvr_geometry *g, const pvr_params *prm, PsfTab *tab)
{
    PsfTab &t = *tab;
    memset(&t, 0, sizeof t);
    t.kxy = prm->psf_kxy;
    t.kz = prm->psf_kz;
    const double to_sigma = 1.0 / (2.0 * sqrt(2.0 * log(2.0)));
    const double sxy = prm->psf_fwhm_xy * to_sigma;
    // the sinc reaches half its peak at u = 0.6033545644: a sinc profile of
    // full width at half maximum F pixels is sinc(1.2067091288 d / F)
    const double sinc_width = 1.2067091288;
    for (int d = -t.kxy; d <= t.kxy; ++d) {
        double v;
        if (prm->psf_kind == PVR_PSF_TAYLOR_SINC)
            v = prm->psf_fwhm_xy > 0.0 ? sinc_series(sinc_width * d / prm->psf_fwhm_xy, prm->psf_sinc_eps)
                                       : (d == 0);
        else
            v = sxy > 0.0 ? exp(-(double)(d * d) / (2.0 * sxy * sxy)) : (d == 0);
        t.gxy[d + t.kxy] = (float)v;
    }
    for (int s = 0; s < g->n_stacks; ++s) {
        const double sz = g->thickness[s] * to_sigma;
        for (int z = -t.kz; z <= t.kz; ++z) {
            const double o = z * prm->psf_dz;
            t.gz[s][z + t.kz] = (float)(sz > 0.0 ? exp(-(o * o) / (2.0 * sz * sz)) : (z == 0));
        }
    }
}

// Checks of a geometry and the PSF / pose settings shared by every entry
// point that takes them (context creation and the context-free forward
// model); returns null when valid, else a one-line reason.
const char *validate_setup(const pvr_geometry *g, const pvr_params *prm)
{
    if (g->nx < 2 || g->ny < 2 || g->nz < 2 || g->nx > 2048 || g->ny > 2048 || g->nz > 2048)
        return "volume sizes must be 2..2048";
    if ((int64_t)g->nx * g->ny * g->nz >= ((int64_t)1 << 31)) return "the volume must have fewer than 2^31 voxels";
    if (g->n_stacks < 1 || g->n_stacks > PVR_MAX_STACKS) return "n_stacks outside 1..16";
    for (int s = 0; s < g->n_stacks; ++s) {
        if (g->stack_w[s] < 1 || g->stack_h[s] < 1 || g->stack_k[s] < 1) return "empty stack";
        if (!(g->thickness[s] >= 0.0) || !isfinite(g->thickness[s])) return "bad slice thickness";
        for (int i = 0; i < 12; ++i)
            if (!isfinite(g->pixel_to_world[s][i])) return "non-finite pixel_to_world";
        const double *S = g->pixel_to_world[s];
        if (!(S[2] * S[2] + S[6] * S[6] + S[10] * S[10] > 0.0)) return "zero slice axis";
    }
    for (int i = 0; i < 12; ++i)
        if (!isfinite(g->world_to_voxel[i])) return "non-finite world_to_voxel";
    if (prm->psf_kxy < 0 || prm->psf_kxy > PVR_MAX_KXY) return "psf_kxy outside 0..3";
    if (prm->psf_kz < 0 || prm->psf_kz > PVR_MAX_KZ) return "psf_kz outside 0..8";
    if (!(prm->psf_dz > 0.0) || !isfinite(prm->psf_dz) || !(prm->psf_fwhm_xy >= 0.0) || !isfinite(prm->psf_fwhm_xy))
        return "bad PSF size";
    if (prm->psf_kind != PVR_PSF_GAUSSIAN && prm->psf_kind != PVR_PSF_TAYLOR_SINC) return "bad psf_kind";
    if (prm->psf_kind == PVR_PSF_TAYLOR_SINC && !(prm->psf_sinc_eps > 0.0 && prm->psf_sinc_eps < 1.0))
        return "psf_sinc_eps outside (0, 1)";
    if (prm->n_params != 6 && prm->n_params != 12) return "n_params must be 6 (rigid) or 12 (affine)";
    if (!(prm->sr_lambda >= 0.0 && prm->sr_lambda <= 1.0)) return "sr_lambda outside 0..1";
    if (prm->sr_lambda > 0.0 && !(prm->sr_edge_delta > 0.0 && isfinite(prm->sr_edge_delta)))
        return "sr_edge_delta must be positive";
    return nullptr;
}

int ctx_n_params(const pvr_ctx *c) { return c->prm.n_params; }

const DevGeom *ctx_dev_geom(const pvr_ctx *c) { return c->d_geom; }

}  // namespace pvr

extern "C" {


void pvr_params_default(pvr_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->psf_fwhm_xy = 1.2;
    p->psf_kxy = 1;
    p->psf_kz = 3;
    p->psf_dz = 1.0;
    p->alpha = 1.0;
    p->conf_eps = 1e-6;
    p->em_c0 = 0.9;
    p->em_sigma_floor_rel = 1e-3;
    p->em_min_valid_frac = 0.1;
    p->patch_rule = 0;
    p->patch_threshold = 0.5;
    p->patch_em_iters = 5;
    p->n_params = 6;
    p->reg_evals = 40;
    p->reg_delta0 = 2.0;
    p->reg_delta_min = 0.01;
    p->reg_grow = 1.0;
    p->reg_fixed_step = 0;
    p->reg_min_valid = 16;
    p->n_sr = 1;
    p->max_patches = 65536;
    p->max_pixels = (int64_t)1 << 27;
    p->max_patch_side = 128;
    p->psf_kind = PVR_PSF_GAUSSIAN;
    p->psf_sinc_eps = 1e-12;
    p->slic_a_min = 0;
    p->sr_lambda = 0.0;
    p->sr_edge_delta = 100.0;
}

int pvr_ctx_create(pvr_ctx **out, const pvr_geometry *g, const pvr_params *prm)
{
    if (!out) return PVR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!g || !prm) return PVR_ERR_INVALID_ARG;
    pvr_ctx *c = new pvr_ctx();
    auto bad = [&](const char *msg) {
        fprintf(stderr, "pvr_ctx_create: %s\n", msg);
        delete c;
        return PVR_ERR_INVALID_ARG;
    };
    if (const char *why = validate_setup(g, prm)) return bad(why);
    if (prm->max_patches < 1 || prm->max_pixels < 1) return bad("capacity must be positive");
    if (prm->max_patch_side < 1 || prm->max_patch_side > kMaxSideLimit)
        return bad("max_patch_side outside 1..256");
    if (prm->patch_em_iters < 0 || prm->reg_evals < 0 || prm->n_sr < 0) return bad("negative count");
    if (prm->slic_a_min != 0 && prm->slic_a_min < 2) return bad("slic_a_min must be 0 or >= 2");
    c->geom = *g;
    c->prm = *prm;
    cudaGetDevice(&c->device);

    // device geometry
    DevGeom &hg = c->hgeom;
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
    c->stack_total = off;
    c->nvox = (int64_t)g->nx * g->ny * g->nz;

    // PSF tables: float64 weights rounded to float32
    make_psf_tab(g, prm, &c->psf);

    // scratch
    Tiling tl = make_tiling(prm->max_patch_side);
    c->tpp_cap = tl.tpp;
    // partial-sum slots also cover the 32-pixel tiling the planner may pick
    // (offered for patch sides up to 128)
    c->tpp_alloc = tl.tpp;
    if (prm->max_patch_side <= 128) {
        int t32 = (prm->max_patch_side + 31) / 32;
        if (t32 * t32 > c->tpp_alloc) c->tpp_alloc = t32 * t32;
    }
    size_t P = (size_t)prm->max_patches, NP = (size_t)prm->max_pixels;
    size_t slots = P * (size_t)c->tpp_alloc * kPartStride;
    c->keep_cap = (int64_t)(P * 4 > (1u << 20) ? P * 4 : (1u << 20));
    cudaError_t e = cudaSuccess;
#define ALLOC(ptr, n) if (e == cudaSuccess) e = dalloc(&(ptr), (n))
    ALLOC(c->d_geom, 1);
    ALLOC(c->fix, P * kFixStride);
    ALLOC(c->part, slots);
    ALLOC(c->epart, P * kPartStride);
    ALLOC(c->gpart, P * (size_t)c->tpp_alloc * kGradStride);
    ALLOC(c->plan_items, P * (size_t)c->tpp_alloc);
    ALLOC(c->plan_counter, 4);
    ALLOC(c->plan_order, P);
    ALLOC(c->pstat, 8);
    ALLOC(c->pbar, P);
    ALLOC(c->wsc, P);
    ALLOC(c->emblk, 512 * 8);
    ALLOC(c->emcount, 1);
    ALLOC(c->ncc_counter, 1);
    ALLOC(c->elig, P);
    ALLOC(c->err, 1);
    ALLOC(c->best, P * kRegStride);
    ALLOC(c->gbest, P * kRegStride);
    ALLOC(c->nbest, P);
    ALLOC(c->trial, P * 12);
    ALLOC(c->delta, P);
    ALLOC(c->ncc_tmp, P);
    ALLOC(c->grad_tmp, P * 12);
    ALLOC(c->active, P);
    ALLOC(c->s_buf, NP);
    ALLOC(c->e_buf, NP);
    ALLOC(c->p_buf, NP);
    ALLOC(c->v_buf, NP);
    ALLOC(c->valid_buf, NP);
    ALLOC(c->mask_tmp, P);
    ALLOC(c->acc2, (size_t)c->nvox);
    ALLOC(c->quad, (size_t)c->nvox);
    if (prm->sr_lambda > 0.0) ALLOC(c->x_next, (size_t)c->nvox);
    {
        // gradient scratch: all tiles if they fit in 2.5 GB, else chunks of whole patches
        size_t per = ncc_gbuf_floats_per_tile(tl, prm->psf_kxy) * sizeof(float);
        long long want = (long long)P * tl.tpp, cap = (long long)((size_t)2560 << 20) / (long long)per;
        if (cap < tl.tpp) cap = tl.tpp;
        c->gbuf_tiles = want < cap ? want : cap;
        ALLOC(c->gbuf, (size_t)c->gbuf_tiles * per / sizeof(float));
    }
    ALLOC(c->keep, (size_t)c->keep_cap);
    ALLOC(c->imax_key, 1);
    ALLOC(c->counts, 4);
    c->n_slices = 0;
    for (int s = 0; s < g->n_stacks; ++s) c->n_slices += g->stack_k[s];
    ALLOC((char *&)c->slice_scr, patches_slice_scratch_bytes(c->n_slices));
    if (prm->slic_a_min > 0) ALLOC((char *&)c->slic_scr, slic_scratch_bytes(*g, prm->slic_a_min, off));
    ALLOC(c->metric_scr, kMetricScratch);
#undef ALLOC
    if (e == cudaSuccess) e = cudaMemcpy(c->d_geom, &hg, sizeof hg, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->err, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(c->emcount, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->acc2, 0, (size_t)c->nvox * sizeof(float2));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        fprintf(stderr, "pvr_ctx_create: %s\n", cudaGetErrorString(e));
        free_all(c);
        delete c;
        return PVR_ERR_CUDA;
    }
    *out = c;
    return PVR_OK;
}

int pvr_ctx_destroy(pvr_ctx *c)
{
    if (!c) return PVR_OK;
    cudaDeviceSynchronize();
    free_all(c);
    for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
    delete c;
    return PVR_OK;
}

const char *pvr_last_error(const pvr_ctx *c) { return c ? c->last_error.c_str() : "null context"; }

int64_t pvr_launch_count(const pvr_ctx *c) { return c ? c->launches : 0; }

int pvr_device_status(pvr_ctx *c, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, c->err, sizeof h, cudaMemcpyDeviceToHost, st), "read error word");
    CUDA_TRY(cudaStreamSynchronize(st), "synchronise");
    CUDA_TRY(cudaMemsetAsync(c->err, 0, sizeof h, st), "clear error word");
    if (h & 1) return fail(c, PVR_ERR_BOUNDS, "a patch row lies outside its stack or pixel range");
    if (h & 2) return fail(c, PVR_ERR_NUMERIC, "a pose produced a non-finite sample map");
    if (h & 4) return fail(c, PVR_ERR_TIMEOUT, "a bounded device wait gave up (tile staging)");
    return PVR_OK;
}

int pvr_patches_build_sizes(pvr_ctx *c, const float *stacks, const int32_t *slice_a,
                            const int32_t *slice_stride, double fg_frac, double keep_frac,
                            int32_t *desc_out, int32_t max_out, int32_t *n_out, int64_t *n_pix_out,
                            void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    REQUIRE(stacks && slice_a && slice_stride && desc_out && n_out && n_pix_out, "NULL argument");
    REQUIRE(max_out >= 0, "max_out < 0");
    REQUIRE(isfinite(fg_frac) && isfinite(keep_frac), "non-finite level");
    int64_t n_cand = 0, pix = 0;
    int gk = 0;
    for (int s = 0; s < c->geom.n_stacks; ++s) {
        const int W = c->geom.stack_w[s], H = c->geom.stack_h[s];
        for (int k = 0; k < c->geom.stack_k[s]; ++k, ++gk) {
            const int a = slice_a[gk], stride = slice_stride[gk];
            REQUIRE(a >= 1 && stride >= 1 && a <= c->prm.max_patch_side,
                    "slice %d: a must be 1..max_patch_side, stride >= 1", gk);
            int64_t nx = W >= a ? (W - a) / stride + 1 : 0, ny = H >= a ? (H - a) / stride + 1 : 0;
            n_cand += nx * ny;
            pix += nx * ny * (int64_t)a * a;
        }
    }
    REQUIRE(n_cand <= c->keep_cap, "%lld candidate patches exceed the scratch (%lld)",
            (long long)n_cand, (long long)c->keep_cap);
    REQUIRE(pix < ((int64_t)1 << 31), "pixel offsets would exceed int32");
    cudaStream_t st = (cudaStream_t)stream;
    int64_t nc = 0;
    CUDA_TRY(launch_patches_build(c->d_geom, c->geom, stacks, c->stack_total, slice_a, slice_stride,
                                  fg_frac, keep_frac, desc_out, max_out, c->keep, &nc, c->imax_key,
                                  c->counts, c->slice_scr, st),
             "patches_build");
    c->launches += nc > 0 ? 3 : 1;
    int32_t h[4];
    CUDA_TRY(cudaMemcpyAsync(h, c->counts, sizeof h, cudaMemcpyDeviceToHost, st), "read counts");
    CUDA_TRY(cudaStreamSynchronize(st), "synchronise");
    *n_out = h[0];
    *n_pix_out = ((int64_t)(uint32_t)h[1]) | ((int64_t)h[2] << 32);
    return PVR_OK;
}

int pvr_patches_build_slic(pvr_ctx *c, const float *stacks, int32_t a, double compactness, int32_t gamma,
                           int32_t n_iter, double fg_frac, double keep_frac, int32_t *desc_out, uint8_t *member_out,
                           int32_t max_out, int32_t *n_out, int64_t *n_pix_out, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    REQUIRE(stacks && desc_out && member_out && n_out && n_pix_out, "NULL argument");
    REQUIRE(a >= 2 && gamma >= 0 && gamma <= 32 && n_iter >= 1 && n_iter <= 100, "a >= 2, gamma 0..32, n_iter 1..100");
    REQUIRE(c->slic_scr != nullptr, "the context has no superpixel scratch (create it with slic_a_min > 0)");
    REQUIRE(a >= c->prm.slic_a_min, "superpixel size %d below the context's slic_a_min %d", a, c->prm.slic_a_min);
    REQUIRE(compactness > 0.0 && isfinite(compactness), "compactness must be positive");
    REQUIRE(max_out >= 0, "max_out < 0");
    REQUIRE(isfinite(fg_frac) && isfinite(keep_frac), "non-finite level");
    const int max_side = c->prm.max_patch_side < 128 ? c->prm.max_patch_side : 128;
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemsetAsync(c->counts, 0, 4 * sizeof(int32_t), st), "clear counts");
    CUDA_TRY(launch_stack_max(stacks, c->stack_total, c->imax_key, st), "stack max");
    int64_t nc = 0;
    CUDA_TRY(launch_patches_build_slic(c->d_geom, c->geom, stacks, c->stack_total, a, compactness, gamma, n_iter,
                                       fg_frac, keep_frac, max_side, desc_out, max_out, member_out,
                                       c->prm.max_pixels, c->imax_key, c->counts, &nc, c->slic_scr, st),
             "patches_build_slic");
    c->launches += 2 + 2 * (int64_t)n_iter + 4;
    int32_t h[4];
    CUDA_TRY(cudaMemcpyAsync(h, c->counts, sizeof h, cudaMemcpyDeviceToHost, st), "read counts");
    CUDA_TRY(cudaStreamSynchronize(st), "synchronise");
    *n_out = h[0];
    *n_pix_out = ((int64_t)(uint32_t)h[1]) | ((int64_t)h[2] << 32);
    REQUIRE(*n_pix_out <= c->prm.max_pixels, "superpixel patches need %lld pixels, above max_pixels",
            (long long)*n_pix_out);
    return PVR_OK;
}

int pvr_patches_build(pvr_ctx *c, const float *stacks, int32_t a, int32_t stride, double fg_frac,
                      double keep_frac, int32_t *desc_out, int32_t max_out, int32_t *n_out,
                      int64_t *n_pix_out, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    std::vector<int32_t> sa((size_t)c->n_slices, a), ss((size_t)c->n_slices, stride);
    return pvr_patches_build_sizes(c, stacks, sa.data(), ss.data(), fg_frac, keep_frac, desc_out,
                                   max_out, n_out, n_pix_out, stream);
}

int pvr_patches_gather(pvr_ctx *c, const float *stacks, const pvr_patches *pp, float *y, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    int ms = 0;
    int rc = check_patches(c, pp, &ms);
    if (rc) return rc;
    REQUIRE(stacks && y, "NULL argument");
    CUDA_TRY(launch_patches_gather(c->d_geom, stacks, pp->desc, pp->n, pp->n_pix, c->err, y,
                                   (cudaStream_t)stream),
             "patches_gather");
    c->launches += pp->n > 0;
    return PVR_OK;
}

int pvr_pose_to_fixed(pvr_ctx *c, const pvr_patches *pp, const double *poses, int32_t *fix,
                      void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    int ms = 0;
    int rc = check_patches(c, pp, &ms);
    if (rc) return rc;
    REQUIRE(pp->n == 0 || (poses && fix), "NULL argument");
    CUDA_TRY(launch_pose_to_fixed(c->d_geom, pp->desc, poses, c->prm.n_params, pp->n, pp->n_pix, ms,
                                  c->psf.kxy, c->psf.kz, fix, c->err, (cudaStream_t)stream),
             "pose_to_fixed");
    c->launches += pp->n > 0;
    return PVR_OK;
}

int pvr_simulate(pvr_ctx *c, const float *x, const pvr_patches *pp, const double *poses, float *sim,
                 uint8_t *valid, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    int ms = 0;
    int rc = check_patches(c, pp, &ms);
    if (rc) return rc;
    REQUIRE(pp->n == 0 || (x && poses && sim && valid), "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    if (pp->n == 0) return PVR_OK;
    if ((rc = pose_fixed(c, pp, ms, poses, st))) return rc;
    if ((rc = build_quad(c, x, st))) return rc;
    Tiling tl = tiling_for(c, ms, pp);
    WorkQueue wqs;
    const WorkQueue *wq = plan_for(c, pp, ms, &tl, &wqs);
    CUDA_TRY_T(PVR_K_SIMULATE, launch_simulate(c->d_geom, c->psf, tl, c->geom.nx, c->geom.ny, c->geom.nz, x,
                                               c->quad, pp->desc, c->fix, pp->n, nullptr, sim, valid,
                                               nullptr, st, wq),
             "simulate");
    c->launches += pp->n > 0;
    return PVR_OK;
}

int pvr_adjoint(pvr_ctx *c, const pvr_patches *pp, const double *poses, const float *r,
                const float *w, float *addon, float *conf, int32_t accumulate, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    int ms = 0;
    int rc = check_patches(c, pp, &ms);
    if (rc) return rc;
    REQUIRE(addon || conf, "addon and conf are both NULL");
    REQUIRE(pp->n == 0 || poses, "NULL poses");
    cudaStream_t st = (cudaStream_t)stream;
    // scatter into the context's interleaved pair accumulator (one vector
    // reduction per voxel corner), then copy / add into the caller's arrays
    CUDA_TRY(cudaMemsetAsync(c->acc2, 0, (size_t)c->nvox * sizeof(float2), st), "clear");
    if ((rc = pose_fixed(c, pp, ms, poses, st))) return rc;
    Tiling tl = tiling_for(c, ms, pp);
    WorkQueue wqs;
    const WorkQueue *wq = plan_for(c, pp, ms, &tl, &wqs);
    CUDA_TRY_T(PVR_K_ADJOINT, launch_adjoint(c->psf, tl, c->geom.nx, c->geom.ny, c->geom.nz, pp->desc, c->fix, pp->n,
                            r, w, nullptr, (float *)c->acc2, nullptr, 1, st, wq),
             "adjoint");
    CUDA_TRY(launch_split_pairs(c->acc2, c->nvox, addon, conf, accumulate, st), "split");
    c->launches += (pp->n > 0) + 1;
    return PVR_OK;
}

int pvr_em_weights(pvr_ctx *c, const float *y, const float *sim, const uint8_t *valid,
                   const pvr_patches *pp, double *state, const uint8_t *mask_in, uint8_t *mask_out,
                   float *p, float *w_patch, float *pbar, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    int ms = 0;
    int rc = check_patches(c, pp, &ms);
    if (rc) return rc;
    REQUIRE(y && valid && state && mask_out && p, "NULL argument");
    REQUIRE(mask_in != mask_out, "mask_in and mask_out must not alias");
    cudaStream_t st = (cudaStream_t)stream;
    Tiling tl = tiling_for(c, ms, pp);
    CUDA_TRY_T(PVR_K_EM, launch_em_stats(y, sim, valid, pp->desc, pp->n, pp->n_pix, tl, c->err, c->part, st),
             "em_stats");
    CUDA_TRY_T(PVR_K_EM, launch_em(y, sim, valid, pp->desc, pp->n, pp->n_pix, tl, c->err, state, mask_in,
                       mask_out, p, w_patch, pbar, c->part, c->pstat, c->pbar, c->wsc, c->elig,
                       c->emblk, c->emcount, c->prm, st),
             "em");
    c->launches += (pp->n > 0) + em_launch_count(pp->n, c->prm);
    return PVR_OK;
}

int pvr_volume_update(pvr_ctx *c, float *x, float *addon, float *conf, int32_t clear, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    REQUIRE(x && addon && conf, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    const float alpha = (float)c->prm.alpha, eps = (float)c->prm.conf_eps;
    if (c->prm.sr_lambda <= 0.0) {
        CUDA_TRY(launch_volume_update(x, addon, conf, c->nvox, alpha, eps, clear, 0, st), "volume_update");
        c->launches += 1;
        return PVR_OK;
    }
    CUDA_TRY(launch_volume_update(x, addon, conf, c->nvox, alpha, eps, 0, 0, st), "volume_update");
    CUDA_TRY(launch_sr_diffuse_split(x, addon, conf, clear, c->x_next, c->geom.nx, c->geom.ny, c->geom.nz,
                                     (float)c->prm.sr_lambda, (float)c->prm.sr_edge_delta, eps, c->err, st),
             "sr_diffuse");
    CUDA_TRY(cudaMemcpyAsync(x, c->x_next, (size_t)c->nvox * sizeof(float), cudaMemcpyDeviceToDevice, st),
             "copy regularised volume");
    c->launches += 2;
    return PVR_OK;
}

int pvr_volume_init(pvr_ctx *c, float *x, const float *y, const pvr_patches *pp,
                    const double *poses, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    int ms = 0;
    int rc = check_patches(c, pp, &ms);
    if (rc) return rc;
    REQUIRE(x && y && (pp->n == 0 || poses), "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemsetAsync(c->acc2, 0, (size_t)c->nvox * sizeof(float2), st), "clear");
    if ((rc = pose_fixed(c, pp, ms, poses, st))) return rc;
    Tiling tl = tiling_for(c, ms, pp);
    CUDA_TRY_T(PVR_K_ADJOINT, launch_adjoint(c->psf, tl, c->geom.nx, c->geom.ny, c->geom.nz, pp->desc, c->fix, pp->n,
                            y, nullptr, nullptr, (float *)c->acc2, nullptr, 1, st),
             "adjoint");
    CUDA_TRY_T(PVR_K_UPDATE, launch_volume_update_pairs(x, c->acc2, c->nvox, 1.0f, (float)c->prm.conf_eps, 1, 1,
                                  st),
             "volume_init");
    c->launches += (pp->n > 0) + 1;
    return PVR_OK;
}

int pvr_patch_metrics(pvr_ctx *c, const float *y, const float *sim, const uint8_t *valid,
                      const pvr_patches *pp, int32_t w, double *out, float *map, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    int ms = 0;
    int rc = check_patches(c, pp, &ms);
    if (rc) return rc;
    REQUIRE(w >= 0 && w <= 16, "window half-width must be 0..16");
    REQUIRE(pp->n == 0 || (y && sim && valid && out), "NULL argument");
    CUDA_TRY(launch_patch_metrics(y, sim, valid, pp->desc, pp->n, w, ms, out, map, (cudaStream_t)stream),
             "patch_metrics");
    c->launches += pp->n > 0;
    return PVR_OK;
}

int pvr_rigidity_map(pvr_ctx *c, const pvr_patches *pp, const double *poses, const float *p,
                     const float *pbar, float *out, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    int ms = 0;
    int rc = check_patches(c, pp, &ms);
    if (rc) return rc;
    REQUIRE(out && (pp->n == 0 || (poses && p && pbar)), "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemsetAsync(c->acc2, 0, (size_t)c->nvox * sizeof(float2), st), "clear");
    if ((rc = pose_fixed(c, pp, ms, poses, st))) return rc;
    Tiling tl = tiling_for(c, ms, pp);
    CUDA_TRY_T(PVR_K_ADJOINT, launch_adjoint(c->psf, tl, c->geom.nx, c->geom.ny, c->geom.nz, pp->desc, c->fix,
                                             pp->n, p, nullptr, nullptr, (float *)c->acc2, nullptr, 1, st,
                                             nullptr, pbar),
               "adjoint");
    CUDA_TRY_T(PVR_K_UPDATE, launch_volume_update_pairs(out, c->acc2, c->nvox, 1.0f, (float)c->prm.conf_eps, 1, 1,
                                                        st),
               "rigidity");
    c->launches += (pp->n > 0) + 1;
    return PVR_OK;
}

int pvr_ncc_grad(pvr_ctx *c, const float *x, const float *y, const pvr_patches *pp,
                 const double *poses, double *ncc, double *grad, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    int ms = 0;
    int rc = check_patches(c, pp, &ms);
    if (rc) return rc;
    REQUIRE(pp->n == 0 || (x && y && poses && ncc), "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    if (pp->n == 0) return PVR_OK;
    if ((rc = pose_fixed(c, pp, ms, poses, st))) return rc;
    if ((rc = build_quad(c, x, st))) return rc;
    Tiling tl = tiling_for(c, ms, pp);
    CUDA_TRY_T(PVR_K_NCC, launch_ncc_grad(c->d_geom, c->psf, tl, c->geom.nx, c->geom.ny, c->geom.nz, x, c->quad, y,
                             pp->desc, c->fix, poses, pp->n, c->s_buf, c->v_buf, c->part,
                             grad ? c->gpart : nullptr, nullptr, c->prm.reg_min_valid, c->gbuf,
                             c->gbuf_tiles, c->ncc_counter, st),
             "ncc_grad");
    CUDA_TRY_T(PVR_K_NCC_FINISH, launch_ncc_finish(c->d_geom, pp->desc, poses, c->prm.n_params, pp->n, tl, c->part,
                                                   c->gpart, c->prm.reg_min_valid, ncc, grad, st),
             "ncc_finish");
    c->launches += ncc_launch_count(tl, pp->n, grad != nullptr, c->gbuf_tiles) + (pp->n > 0);
    return PVR_OK;
}

int pvr_pose_grad(pvr_ctx *c, const float *x, const float *r, const pvr_patches *pp,
                  const double *poses, double *grad, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    int ms = 0;
    int rc = check_patches(c, pp, &ms);
    if (rc) return rc;
    REQUIRE(pp->n == 0 || (x && r && poses && grad), "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    if (pp->n == 0) return PVR_OK;
    if ((rc = pose_fixed(c, pp, ms, poses, st))) return rc;
    Tiling tl = tiling_for(c, ms, pp);
    CUDA_TRY_T(PVR_K_NCC, launch_pose_vjp(c->psf, tl, c->geom.nx, c->geom.ny, c->geom.nz, x, r,
                                          pp->desc, c->fix, pp->n, c->gpart, c->gbuf, c->gbuf_tiles,
                                          c->ncc_counter, st),
               "pose_vjp");
    CUDA_TRY_T(PVR_K_NCC_FINISH, launch_ncc_finish(c->d_geom, pp->desc, poses, c->prm.n_params, pp->n, tl, nullptr,
                                                   c->gpart, c->prm.reg_min_valid, nullptr, grad, st),
               "pose_vjp_finish");
    c->launches += 2;
    return PVR_OK;
}

// Registration rounds; gathers from c->quad, which the caller has built from x.
// keep_best: for one-tile patches, the NCC kernels also leave the forward
// model at each patch's best pose in e_buf, valid_buf and epart (BestSim);
// *kept tells whether they did.
static int register_impl(pvr_ctx *c, const float *x, const float *y, const pvr_patches *pp, int ms,
                         double *poses, int n_evals, double *ncc_out, cudaStream_t st,
                         bool keep_best = false, bool *kept = nullptr)
{
    int n = pp->n;
    if (kept) *kept = false;
    if (n == 0 || n_evals <= 0) return PVR_OK;
    Tiling tl = tiling_for(c, ms, pp);
    keep_best = keep_best && tl.tpp == 1;
    BestSim bs;
    bs.nbest = c->nbest;
    bs.fixed = c->prm.reg_fixed_step != 0;
    if (keep_best) {
        bs.mode = 1;
        bs.e = c->e_buf;
        bs.valid = c->valid_buf;
        bs.part = c->epart;
    }
    CUDA_TRY(launch_reg_init(poses, c->prm.n_params, n, c->best, c->trial, c->delta, c->active,
                             c->prm.reg_delta0, st),
             "reg_init");
    c->launches += 1;
    for (int ev = 0; ev < n_evals; ++ev) {
        int rc = pose_fixed(c, pp, ms, c->trial, st);
        if (rc) return rc;
        // the last evaluation only decides acceptance: its gradient would
        // never be used, so it computes the NCC alone
        const bool need_grad = ev < n_evals - 1;
        double *gpart = need_grad ? c->gpart : nullptr, *grad = need_grad ? c->grad_tmp : nullptr;
        CUDA_TRY_T(PVR_K_NCC, launch_ncc_grad(c->d_geom, c->psf, tl, c->geom.nx, c->geom.ny, c->geom.nz, x, c->quad, y,
                                 pp->desc, c->fix, c->trial, n, c->s_buf, c->v_buf, c->part,
                                 gpart, c->active, c->prm.reg_min_valid, c->gbuf, c->gbuf_tiles,
                                 c->ncc_counter, st, bs),
                 "ncc_grad");
        if (keep_best) bs.mode = 2;   // after the first evaluation: accepted trials only
        bs.grad_if_accepted = 1;      // later evaluations: gradients of accepted trials only
        CUDA_TRY_T(PVR_K_NCC_FINISH, launch_ncc_finish(c->d_geom, pp->desc, c->trial, c->prm.n_params, n, tl, c->part,
                                                       gpart, c->prm.reg_min_valid, c->ncc_tmp, grad, st),
                 "ncc_finish");
        CUDA_TRY_T(PVR_K_REG_STEP, launch_reg_step(c->d_geom, pp->desc, n, ev, ev == n_evals - 1, c->ncc_tmp,
                                 grad, c->best, c->gbest, c->nbest, c->trial, c->delta,
                                 c->active, c->prm, st),
                 "reg_step");
        c->launches += ncc_launch_count(tl, n, need_grad, c->gbuf_tiles) + 2;
    }
    CUDA_TRY(launch_reg_finish(c->best, c->nbest, c->prm.n_params, n, poses, ncc_out, st), "reg_finish");
    c->launches += 1;
    if (kept) *kept = keep_best;
    return PVR_OK;
}

int pvr_register(pvr_ctx *c, const float *x, const float *y, const pvr_patches *pp, double *poses,
                 int32_t n_evals, double *ncc, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    int ms = 0;
    int rc = check_patches(c, pp, &ms);
    if (rc) return rc;
    REQUIRE(n_evals >= 0, "n_evals < 0");
    REQUIRE(pp->n == 0 || (x && y && poses), "NULL argument");
    if (pp->n == 0 || n_evals == 0) return PVR_OK;
    if ((rc = build_quad(c, x, (cudaStream_t)stream))) return rc;
    return register_impl(c, x, y, pp, ms, poses, n_evals, ncc, (cudaStream_t)stream);
}

int pvr_reconstruct_iter(pvr_ctx *c, float *x, const float *y, const pvr_patches *pp, double *poses,
                         double *state, uint8_t *mask, float *p, float *w_patch, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    int ms = 0;
    int rc = check_patches(c, pp, &ms);
    if (rc) return rc;
    REQUIRE(x && y && state && mask && (pp->n == 0 || poses), "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = build_quad(c, x, st))) return rc;
    // one-tile patches under the super-resolution tiling too: the
    // registration's NCC kernels keep the forward model at the final poses,
    // and the first pass below reuses it instead of simulating again
    Tiling tl = tiling_for(c, ms, pp);
    WorkQueue wqs;
    const WorkQueue *wq = plan_for(c, pp, ms, &tl, &wqs);
    bool kept = false;
    if ((rc = register_impl(c, x, y, pp, ms, poses, c->prm.reg_evals, nullptr, st, tl.tpp == 1, &kept)))
        return rc;
    if ((rc = pose_fixed(c, pp, ms, poses, st))) return rc;
    CUDA_TRY(cudaMemsetAsync(c->acc2, 0, (size_t)c->nvox * sizeof(float2), st), "clear");
    for (int it = 0; it < c->prm.n_sr; ++it) {
        // x changes with every SR pass: refresh its quad copy after the first
        if (it > 0 && (rc = build_quad(c, x, st))) return rc;
        // first pass after a registration that kept the forward model: the
        // residuals, valid flags and EM partials are already in place
        const bool reuse = it == 0 && kept;
        double *part = reuse ? c->epart : c->part;
        if (!reuse) {
            // the work queue visits non-empty tiles only: empty slots of the
            // EM partials must read as zero
            if (wq)
                CUDA_TRY(cudaMemsetAsync(c->part, 0, (size_t)pp->n * tl.tpp * kPartStride * sizeof(double), st),
                         "clear partials");
            CUDA_TRY_T(PVR_K_SIMULATE, launch_simulate(c->d_geom, c->psf, tl, c->geom.nx, c->geom.ny, c->geom.nz, x,
                                                       c->quad, pp->desc, c->fix, pp->n, y, c->e_buf,
                                                       c->valid_buf, c->part, st, wq),
                     "simulate");
        }
        CUDA_TRY_T(PVR_K_EM, launch_em(c->e_buf, nullptr, c->valid_buf, pp->desc, pp->n, pp->n_pix, tl, c->err,
                           state, mask, c->mask_tmp, c->p_buf, w_patch, nullptr, part, c->pstat,
                           c->pbar, c->wsc, c->elig, c->emblk, c->emcount, c->prm, st),
                 "em");
        CUDA_TRY(cudaMemcpyAsync(mask, c->mask_tmp, (size_t)pp->n, cudaMemcpyDeviceToDevice, st),
                 "mask copy");
        CUDA_TRY_T(PVR_K_ADJOINT, launch_adjoint(c->psf, tl, c->geom.nx, c->geom.ny, c->geom.nz, pp->desc, c->fix,
                                pp->n, c->e_buf, c->p_buf, mask, (float *)c->acc2, nullptr, 1, st, wq),
                 "adjoint");
        int upd = 0;
        if ((rc = sr_update_pairs(c, x, st, &upd))) return rc;
        c->launches += (pp->n > 0 ? (reuse ? 1 : 2) : 0) + upd + em_launch_count(pp->n, c->prm);
    }
    if (p && pp->n_pix > 0)
        CUDA_TRY(cudaMemcpyAsync(p, c->p_buf, (size_t)pp->n_pix * sizeof(float),
                                 cudaMemcpyDeviceToDevice, st),
                 "p copy");
    return PVR_OK;
}

// ------------------------------------------------------------ work plan --

namespace {

// Launch order of a patch table: the patches sorted (stably) by the block of
// 32^3 voxels that holds their centre at the identity pose, z block first,
// then y, then x.  The CTAs running at one time then gather from (and
// scatter to) a compact part of the volume whatever the stack order of the
// table; in table order the patches of each stack sweep the whole volume,
// and the volume data is fetched from DRAM again for every stack.  Rows with
// an invalid stack index keep key 0 (the kernels skip them anyway).
std::vector<int32_t> spatial_patch_order(const pvr_geometry &g, const std::vector<int32_t> &desc, int n)
{
    std::vector<std::pair<int64_t, int32_t>> v((size_t)n);
    const double *W = g.world_to_voxel;
    for (int p = 0; p < n; ++p) {
        const int32_t *d = &desc[8 * (size_t)p];
        int64_t key = 0;
        if (d[0] >= 0 && d[0] < g.n_stacks) {
            const double *M = g.pixel_to_world[d[0]];
            const double ci = d[2] + 0.5 * d[4] - 0.5, cj = d[3] + 0.5 * d[5] - 0.5, k = d[1];
            double w[3];
            for (int r = 0; r < 3; ++r) w[r] = M[4 * r] * ci + M[4 * r + 1] * cj + M[4 * r + 2] * k + M[4 * r + 3];
            int64_t b[3];
            for (int r = 0; r < 3; ++r) {
                const double v_ = W[4 * r] * w[0] + W[4 * r + 1] * w[1] + W[4 * r + 2] * w[2] + W[4 * r + 3];
                b[r] = v_ >= 0.0 ? (v_ < 32.0 * 1023.0 ? (int64_t)(v_ / 32.0) : 1023) : 0;   // NaN -> 0
            }
            key = (b[2] * 1024 + b[1]) * 1024 + b[0];
        }
        v[(size_t)p] = {key, (int32_t)p};
    }
    std::stable_sort(v.begin(), v.end(), [](const std::pair<int64_t, int32_t> &a,
                                            const std::pair<int64_t, int32_t> &b) { return a.first < b.first; });
    std::vector<int32_t> order((size_t)n);
    for (int i = 0; i < n; ++i) order[(size_t)i] = v[(size_t)i].second;
    return order;
}

// Non-empty (patch, tile) slots of the table under tiling tl, largest tiles
// first (stable, so equal tiles keep the patch order given).
std::vector<int32_t> tile_items(const std::vector<int32_t> &desc, const std::vector<int32_t> &porder,
                                const Tiling &tl)
{
    std::vector<std::pair<int, int32_t>> v;
    v.reserve(porder.size() * tl.tpp);
    for (const int32_t p : porder) {
        const int w = desc[8 * (size_t)p + 4], h = desc[8 * (size_t)p + 5];
        for (int t = 0; t < tl.tpp; ++t) {
            const int i0 = (t % tl.tiles_x) * tl.T, j0 = (t / tl.tiles_x) * tl.T;
            if (i0 >= w || j0 >= h) continue;
            const int tw = w - i0 < tl.T ? w - i0 : tl.T, th = h - j0 < tl.T ? h - j0 : tl.T;
            v.push_back({tw * th, (int32_t)((int64_t)p * tl.tpp + t)});
        }
    }
    std::stable_sort(v.begin(), v.end(), [](const std::pair<int, int32_t> &a,
                                            const std::pair<int, int32_t> &b) { return a.first > b.first; });
    std::vector<int32_t> items(v.size());
    for (size_t i = 0; i < v.size(); ++i) items[i] = v[i].second;
    return items;
}

}  // namespace

int pvr_plan(pvr_ctx *c, const pvr_patches *pp, const float *x, const float *y, const double *poses,
             int32_t tile, int32_t mode, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    int ms = 0;
    int rc = check_patches(c, pp, &ms);
    if (rc) return rc;
    REQUIRE(tile == 0 || tile == 32 || tile == 64, "tile must be 0 (tune), 32 or 64");
    REQUIRE(mode >= -1 && mode <= 1, "mode must be -1 (tune), 0 or 1");
    const bool autotune = tile == 0 || mode == -1;
    REQUIRE(!autotune || (x && y && poses), "tuning needs x, y and poses");
    cudaStream_t st = (cudaStream_t)stream;
    c->plan_n = -1;   // no plan while this one is being made
    if (pp->n == 0) return PVR_OK;
    std::vector<int32_t> desc((size_t)pp->n * 8);
    CUDA_TRY(cudaMemcpyAsync(desc.data(), pp->desc, desc.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st),
             "read table");
    CUDA_TRY(cudaStreamSynchronize(st), "synchronise");
    const std::vector<int32_t> porder = spatial_patch_order(c->geom, desc, pp->n);
    CUDA_TRY(cudaMemcpyAsync(c->plan_order, porder.data(), porder.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                             st),
             "upload order");
    // candidates: tile side 64 (or the largest side below it), and 32 where
    // the partial buffers hold its slots; each as one CTA per slot or as a
    // persistent work queue
    std::vector<int> sides;
    if (tile != 32) sides.push_back(64);
    if (tile != 64 && (int64_t)((ms + 31) / 32) * ((ms + 31) / 32) <= c->tpp_alloc) sides.push_back(32);
    REQUIRE(!sides.empty(), "32-pixel tiles need max_patch_side <= 128");
    struct Cand {
        Tiling tl;
        int mode;
        std::vector<int32_t> items;
    };
    std::vector<Cand> cands;
    for (int T : sides) {
        Tiling tl = make_tiling_t(ms, T);
        tl.member = pp->member;
        tl.order = c->plan_order;
        if (mode != 0) cands.push_back({tl, 1, tile_items(desc, porder, tl)});
        if (mode != 1) cands.push_back({tl, 0, {}});
    }
    int best = 0;
    if (autotune && cands.size() > 1) {
        if ((rc = pose_fixed(c, pp, ms, poses, st))) return rc;
        if ((rc = build_quad(c, x, st))) return rc;
        cudaEvent_t e0, e1;
        CUDA_TRY(cudaEventCreate(&e0), "event");
        CUDA_TRY(cudaEventCreate(&e1), "event");
        float best_ms = 1e30f;
        for (size_t k = 0; k < cands.size(); ++k) {
            Cand &cd = cands[k];
            WorkQueue wq;
            if (cd.mode == 1) {
                CUDA_TRY(cudaMemcpyAsync(c->plan_items, cd.items.data(), cd.items.size() * sizeof(int32_t),
                                         cudaMemcpyHostToDevice, st),
                         "upload items");
                wq.items = c->plan_items;
                wq.n_items = (int)cd.items.size();
                wq.counter = c->plan_counter;
            }
            float t_sum[3];
            for (int rep = 0; rep < 4; ++rep) {
                CUDA_TRY(cudaEventRecord(e0, st), "event");
                CUDA_TRY(launch_simulate(c->d_geom, c->psf, cd.tl, c->geom.nx, c->geom.ny, c->geom.nz, x,
                                         c->quad, pp->desc, c->fix, pp->n, y, c->e_buf, c->valid_buf,
                                         nullptr, st, cd.mode ? &wq : nullptr),
                         "simulate");
                CUDA_TRY(launch_adjoint(c->psf, cd.tl, c->geom.nx, c->geom.ny, c->geom.nz, pp->desc, c->fix,
                                        pp->n, c->e_buf, nullptr, nullptr, (float *)c->acc2, nullptr, 1, st,
                                        cd.mode ? &wq : nullptr),
                         "adjoint");
                CUDA_TRY(cudaEventRecord(e1, st), "event");
                CUDA_TRY(cudaEventSynchronize(e1), "synchronise");
                float ms_ = 0.f;
                cudaEventElapsedTime(&ms_, e0, e1);
                if (rep > 0) t_sum[rep - 1] = ms_;   // first run warms up
            }
            float med = t_sum[0] + t_sum[1] + t_sum[2] - fminf(t_sum[0], fminf(t_sum[1], t_sum[2])) -
                        fmaxf(t_sum[0], fmaxf(t_sum[1], t_sum[2]));
            if (med < best_ms) {
                best_ms = med;
                best = (int)k;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        CUDA_TRY(cudaMemsetAsync(c->acc2, 0, (size_t)c->nvox * sizeof(float2), st), "clear");
    }
    Cand &cd = cands[best];
    if (cd.mode == 1)
        CUDA_TRY(cudaMemcpyAsync(c->plan_items, cd.items.data(), cd.items.size() * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, st),
                 "upload items");
    CUDA_TRY(cudaStreamSynchronize(st), "synchronise");
    c->plan_tl = cd.tl;
    c->plan_mode = cd.mode;
    c->plan_n_items = (int)cd.items.size();
    c->plan_desc = pp->desc;
    c->plan_n = pp->n;
    c->plan_npix = pp->n_pix;
    return PVR_OK;
}

int pvr_plan_info(const pvr_ctx *c, int32_t *tile, int32_t *mode, int32_t *n_items)
{
    if (!c || !tile || !mode || !n_items) return PVR_ERR_INVALID_ARG;
    const bool on = c->plan_n >= 0;
    *tile = on ? c->plan_tl.T : 0;
    *mode = on ? c->plan_mode : -1;
    *n_items = on ? c->plan_n_items : 0;
    return PVR_OK;
}

int pvr_plan_order(pvr_ctx *c, int32_t *host_out, int32_t n, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    REQUIRE(c->plan_n >= 0, "no plan is held");
    REQUIRE(n == c->plan_n && (n == 0 || host_out), "n must be the planned table's patch count");
    if (n == 0) return PVR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(host_out, c->plan_order, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st),
             "read order");
    CUDA_TRY(cudaStreamSynchronize(st), "synchronise");
    return PVR_OK;
}

int pvr_plan_clear(pvr_ctx *c)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    c->plan_n = -1;
    return PVR_OK;
}

// ---------------------------------------------------------------- graphs --

int pvr_graph_capture(pvr_ctx *c, float *x, const float *y, const pvr_patches *pp, double *poses,
                      double *state, uint8_t *mask, float *p, float *w_patch, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    REQUIRE(stream != nullptr, "capture needs a non-default stream");
    REQUIRE(!c->prof, "disable the profiler before capturing");
    cudaStream_t st = (cudaStream_t)stream;
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
    }
    const int64_t l0 = c->launches;
    CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed), "begin capture");
    int rc = pvr_reconstruct_iter(c, x, y, pp, poses, state, mask, p, w_patch, stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc != PVR_OK) {
        if (g) cudaGraphDestroy(g);
        c->launches = l0;
        return rc;
    }
    CUDA_TRY(e, "end capture");
    e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    cudaGraphDestroy(g);
    CUDA_TRY(e, "instantiate");
    c->graph_launches = c->launches - l0;
    c->launches = l0;
    return PVR_OK;
}

int pvr_graph_launch(pvr_ctx *c, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    REQUIRE(c->graph_exec != nullptr, "no captured graph");
    CUDA_TRY(cudaGraphLaunch(c->graph_exec, (cudaStream_t)stream), "graph launch");
    c->launches += c->graph_launches;
    return PVR_OK;
}

int pvr_profile_enable(pvr_ctx *c, int32_t enable)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    if (enable && c->evpool.empty()) {
        c->evpool.resize(kProfEvents);
        for (size_t i = 0; i < kProfEvents; ++i)
            if (cudaEventCreate(&c->evpool[i]) != cudaSuccess) {
                for (size_t j = 0; j < i; ++j) cudaEventDestroy(c->evpool[j]);
                c->evpool.clear();
                return fail(c, PVR_ERR_CUDA, "cannot create profiler events");
            }
    }
    c->prof = enable != 0;
    return PVR_OK;
}

int pvr_profile_read(pvr_ctx *c, double *ms, int64_t *launches, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    REQUIRE(ms, "NULL argument");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream), "synchronise");
    for (int k = 0; k < PVR_K_N; ++k) {
        ms[k] = 0.0;
        if (launches) launches[k] = 0;
    }
    for (auto &r : c->rec) {
        float t = 0.f;
        CUDA_TRY(cudaEventSynchronize(c->evpool[r.second + 1]), "event");
        CUDA_TRY(cudaEventElapsedTime(&t, c->evpool[r.second], c->evpool[r.second + 1]), "elapsed");
        ms[r.first] += t;
        if (launches) launches[r.first] += 1;
    }
    c->rec.clear();
    c->ev_next = 0;
    return PVR_OK;
}

int pvr_metrics(pvr_ctx *c, const float *ref, const float *img, const uint8_t *mask, int64_t n,
                double *out, void *stream)
{
    if (!c) return PVR_ERR_INVALID_ARG;
    REQUIRE(ref && img && out && n >= 0, "bad argument");
    CUDA_TRY(launch_metrics(ref, img, mask, n, c->metric_scr, out, (cudaStream_t)stream), "metrics");
    c->launches += 3;
    return PVR_OK;
}

}  // extern "C"
