/*
 * pvr_oracle.c -- plain, slow FP64 CPU oracle for the PVR hot path
 * (Alansary et al., "PVR: Patch-to-Volume Reconstruction for Large Area
 * Motion Correction of Fetal MRI", arXiv:1611.07289).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * What it computes, one function per step of the method:
 *   or_patches_build   square patches of side a and stride w      (Sec. II "Patch Extraction")
 *   or_patches_build_sizes  the same with a side and stride per slice (multi-scale patches, Sec. II)
 *   or_pose_fixed      patch pose -> pixel-to-voxel map, Q11.20  (Eq. 1, W_i = D B T_i; Sec. II registration)
 *   or_simulate        Gaussian-PSF forward model of every patch  (Eq. 1; Sec. II "Patch to Volume Registration")
 *   or_adjoint         exact transpose of or_simulate             (super-resolution update, Sec. II)
 *   or_em_weights      voxel/pixel EM robust statistics + patch   (Eqs. for m, p and p-bar, Sec. II "EM-Based
 *                      potentials and patch classification         Outlier Removal")
 *   or_volume_update   weighted SIRT step                         (super-resolution by gradient descent, Sec. II)
 *   or_sr_update       the SIRT step followed by an edge-preserving  (the regularised super-resolution PVR builds
 *                      anisotropic-diffusion step                   on, Sec. I related work, Sec. II)
 *   or_ncc_grad        NCC of a patch and d NCC / d pose          (Sec. II registration with CC; Eq. cross_corr)
 *   or_sim_pose_vjp    d (sum r * sim) / d pose of one patch      (Eq. 1 differentiated through the sample positions)
 *   or_register        per-patch gradient ascent on NCC           (Sec. III "patch-wise gradient descent")
 *   or_metrics         PSNR, CC, SSIM, DSSIM                      (Eqs. cross_corr, PSNR, SSIM, DSSIM)
 *   or_patch_metrics   the same per patch + local DSSIM heat map  (Sec. IV-A patch evaluation)
 *
 * Where the paper is silent (discretisation of the PSF, the fixed-point
 * sample lattice, EM initialisation, the patch classification rule, the
 * optimiser) the readings below are the ones the design document lists.
 *
 * Parity notes.  Integer quantities (patch tables, fixed-point sample
 * positions, in-volume flags, masks) must match the CUDA path bit for bit, so
 * the pose -> fixed-point map is evaluated with plain IEEE double operations
 * in a fixed order, with a sine/cosine written here from their Taylor series
 * (no libm trigonometry), and the file is compiled without FP contraction.
 * Floating-point results are FP64 throughout.
 *
 * Parity unpinned: the patch classification rule (or_em_weights, step 5) has
 * no counterpart printed in the paper; the oracle defines it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_STACKS 16
#define OR_FRAC_BITS 20
#define OR_ONE ((int64_t)1 << OR_FRAC_BITS)
#define OR_FRAC_MASK (OR_ONE - 1)

/* ---------------------------------------------------------------- types -- */

/* Acquisition and reconstruction geometry.  w2v maps world (mm) to volume
 * voxel index (voxel centres at integer indices), p2w[s] maps stack-s pixel
 * coordinates (column, row, slice) to world; both are 3x4 row-major affine
 * matrices whose implied bottom row is (0,0,0,1).  thick[s] is the slice
 * thickness (through-plane FWHM) of stack s in mm. */
typedef struct {
    int nx, ny, nz, n_stacks;
    int sw[OR_MAX_STACKS], sh[OR_MAX_STACKS], sk[OR_MAX_STACKS];
    double w2v[12];
    double p2w[OR_MAX_STACKS][12];
    double thick[OR_MAX_STACKS];
} or_geom;

/* PSF discretisation: in-plane taps at pixel offsets -kxy..kxy,
 * through-plane samples at offsets zeta*dz mm, zeta = -kz..kz.  kind 0:
 * Gaussian in-plane profile; kind 1: sinc in-plane profile evaluated by its
 * Taylor series to relative error eps (Sec. II); the through-plane slice
 * profile is Gaussian in both. */
typedef struct {
    double fwhm_xy;
    int kxy;
    int kz;
    double dz;
    int kind;
    double eps;
} or_psf;

/* EM / patch-classification parameters. */
typedef struct {
    double c0;              /* initial inlier proportion */
    double sigma_floor_rel; /* sigma^2 >= (sigma_floor_rel * range(e))^2 */
    double min_valid_frac;  /* patches with fewer valid pixels are excluded */
    int patch_rule;         /* 0: Gaussian-inlier / uniform-outlier model; 1: threshold */
    double patch_threshold; /* rule 1: inlier iff p-bar >= threshold */
    int patch_em_iters;     /* EM iterations of the patch-level model per call */
} or_em_params;

/* Registration parameters. */
typedef struct {
    int n_params;       /* 6 (rigid) or 12 (affine) */
    int n_eval;         /* NCC evaluations per registration round */
    double delta0;      /* initial step (mm / degrees) */
    double delta_min;   /* stop when the step falls below this */
    int fixed_step;     /* 1: always accept, constant step (parity mode) */
    int min_valid;      /* fewer valid pixels: NCC = 0, no update */
    double grow;        /* step factor after an accepted trial */
} or_reg_params;

/* EM state vector (shared layout with callers; plain doubles). */
enum {
    ST_INIT = 0, ST_SIGMA2, ST_C, ST_M, ST_MU_P, ST_SIGMA2_P, ST_C_P, ST_M_P,
    ST_N_PART, ST_SUM_P, ST_SUM_PE2, ST_EMIN, ST_EMAX, ST_N_ELIG, ST_N_IN,
    ST_SIGMA2_USED, ST_LEN = 16
};

/* ------------------------------------------------------------ utilities -- */

/* sin and cos of an angle in degrees.  Reduction to r in [-45, 45] degrees by
 * the nearest multiple of 90, then the Maclaurin series of sin and cos in
 * nested (Horner) form, truncated after the x^23 / x^22 terms (remainder
 * below 1e-26 for |x| <= pi/4); each nesting step multiplies by the correctly
 * rounded reciprocal of its integer denominator.  Only IEEE +,-,*,/ are used,
 * in a fixed order, so the result is reproducible bit for bit on any IEEE
 * machine. */
static void or_sincos_deg(double deg, double *s_out, double *c_out)
{
    double k = nearbyint(deg / 90.0);
    double r = deg - 90.0 * k;
    double x = r * 0.017453292519943295769;
    double x2 = x * x;
    double ts = 1.0, tc = 1.0;
    for (int n = 11; n >= 1; --n) {
        ts = 1.0 - (x2 * ts) * (1.0 / (double)((2 * n) * (2 * n + 1)));
        tc = 1.0 - (x2 * tc) * (1.0 / (double)((2 * n - 1) * (2 * n)));
    }
    double sr = x * ts, cr = tc;
    long q = ((long)fmod(k, 4.0) + 4) % 4;
    switch (q) {
    case 0: *s_out = sr; *c_out = cr; break;
    case 1: *s_out = cr; *c_out = -sr; break;
    case 2: *s_out = -sr; *c_out = -cr; break;
    default: *s_out = -cr; *c_out = sr; break;
    }
}

/* Linear part of the patch transform.  Rigid: R = Rz(rz) Ry(ry) Rx(rx),
 * angles in degrees, entries written out in closed form.  Affine: I + D. */
static void or_linear_part(const double *th, int n_params, double L[9])
{
    if (n_params == 12) {
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                L[r * 3 + c] = (r == c ? 1.0 : 0.0) + th[3 + r * 3 + c];
        return;
    }
    double sx, cx, sy, cy, sz, cz;
    or_sincos_deg(th[3], &sx, &cx);
    or_sincos_deg(th[4], &sy, &cy);
    or_sincos_deg(th[5], &sz, &cz);
    L[0] = cz * cy;
    L[1] = -(sz * cx) + (cz * sy) * sx;
    L[2] = sz * sx + (cz * sy) * cx;
    L[3] = sz * cy;
    L[4] = cz * cx + (sz * sy) * sx;
    L[5] = -(cz * sx) + (sz * sy) * cx;
    L[6] = -sy;
    L[7] = cy * sx;
    L[8] = cy * cx;
}

/* World position of the centre of a patch's pixel rectangle. */
static void or_patch_centre(const or_geom *g, const int *d, double c[3])
{
    const double *S = g->p2w[d[0]];
    double u = (double)d[2] + (double)(d[4] - 1) * 0.5;
    double v = (double)d[3] + (double)(d[5] - 1) * 0.5;
    double k = (double)d[1];
    for (int r = 0; r < 3; ++r)
        c[r] = ((S[r * 4 + 0] * u + S[r * 4 + 1] * v) + S[r * 4 + 2] * k) + S[r * 4 + 3];
}

/* Full pixel -> voxel map of a patch as a 3x4 matrix: M = W . T(theta) . S,
 * T(w) = L (w - c) + c + t with c the patch centre. */
static void or_patch_matrix(const or_geom *g, const int *d, const double *th, int n_params,
                            double M[12])
{
    const double *S = g->p2w[d[0]];
    const double *W = g->w2v;
    double L[9], c[3], tau[3], A[12];
    or_linear_part(th, n_params, L);
    or_patch_centre(g, d, c);
    for (int r = 0; r < 3; ++r) {
        double Lc = (L[r * 3 + 0] * c[0] + L[r * 3 + 1] * c[1]) + L[r * 3 + 2] * c[2];
        tau[r] = (c[r] + th[r]) - Lc;
    }
    for (int r = 0; r < 3; ++r) {
        for (int col = 0; col < 4; ++col)
            A[r * 4 + col] = (L[r * 3 + 0] * S[0 * 4 + col] + L[r * 3 + 1] * S[1 * 4 + col])
                             + L[r * 3 + 2] * S[2 * 4 + col];
        A[r * 4 + 3] = A[r * 4 + 3] + tau[r];
    }
    for (int r = 0; r < 3; ++r) {
        for (int col = 0; col < 4; ++col)
            M[r * 4 + col] = (W[r * 4 + 0] * A[0 * 4 + col] + W[r * 4 + 1] * A[1 * 4 + col])
                             + W[r * 4 + 2] * A[2 * 4 + col];
        M[r * 4 + 3] = M[r * 4 + 3] + W[r * 4 + 3];
    }
}

/* Scale from one slice-index unit to one through-plane PSF step of dz mm. */
static double or_zeta_scale(const or_geom *g, int stack, double dz)
{
    const double *S = g->p2w[stack];
    double n2 = (S[2] * S[2] + S[6] * S[6]) + S[10] * S[10];
    return dz / sqrt(n2);
}

static int or_quantise(double v, int64_t *out)
{
    if (!isfinite(v)) return 0;
    double s = nearbyint(v * 1048576.0);
    if (!(fabs(s) < 2147483648.0)) return 0;
    *out = (int64_t)s;
    return 1;
}

/* ------------------------------------------------------- pose -> fixed -- */

/* Fixed-point sample lattice of patch d under pose th.
 * f[0..2] = o     : voxel position of patch pixel (0,0) in its slice
 * f[3..5] = e_i   : one pixel step along the patch columns
 * f[6..8] = e_j   : one pixel step along the patch rows
 * f[9..11]= e_z   : one through-plane PSF step of dz mm along the slice normal
 * f[12]   = 1 if the patch's sample box lies inside the representable range,
 *           0 otherwise (then every pixel of the patch is invalid)
 * All in Q11.20 (value * 2^20, round half to even). */
int or_pose_fixed(const or_geom *g, const or_psf *psf, const int *d, const double *th,
                  int n_params, int64_t f[16])
{
    double M[12];
    memset(f, 0, 16 * sizeof(int64_t));
    or_patch_matrix(g, d, th, n_params, M);
    double zs = or_zeta_scale(g, d[0], psf->dz);
    double x0 = (double)d[2], y0 = (double)d[3], k = (double)d[1];
    double fv[12];
    for (int r = 0; r < 3; ++r) {
        fv[r] = ((M[r * 4 + 0] * x0 + M[r * 4 + 1] * y0) + M[r * 4 + 2] * k) + M[r * 4 + 3];
        fv[3 + r] = M[r * 4 + 0];
        fv[6 + r] = M[r * 4 + 1];
        fv[9 + r] = M[r * 4 + 2] * zs;
    }
    int ok = 1;
    for (int i = 0; i < 12; ++i) ok &= or_quantise(fv[i], &f[i]);
    if (ok) {
        int K = psf->kxy, Kz = psf->kz;
        int64_t ci[2] = {-K, d[4] - 1 + K}, cj[2] = {-K, d[5] - 1 + K}, cz[2] = {-Kz, Kz};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int z = 0; z < 2; ++z)
                    for (int r = 0; r < 3; ++r) {
                        int64_t q = f[r] + ci[a] * f[3 + r] + cj[b] * f[6 + r] + cz[z] * f[9 + r];
                        if (q > ((int64_t)1 << 30) || q < -((int64_t)1 << 30)) ok = 0;
                    }
    }
    if (!ok) memset(f, 0, 12 * sizeof(int64_t));
    f[12] = ok;
    return ok;
}

void or_pose_fixed_all(const or_geom *g, const or_psf *psf, const int *desc, const double *poses,
                       int n_params, int P, int64_t *fix)
{
    for (int p = 0; p < P; ++p)
        or_pose_fixed(g, psf, desc + 8 * p, poses + (size_t)n_params * p, n_params,
                      fix + 16 * (size_t)p);
}

/* -------------------------------------------------------------- sampling -- */

/* Position of lattice point (i, j) at through-plane step z. */
static void or_lattice_pos(const int64_t *f, int i, int j, int z, int64_t q[3])
{
    for (int r = 0; r < 3; ++r)
        q[r] = f[r] + (int64_t)i * f[3 + r] + (int64_t)j * f[6 + r] + (int64_t)z * f[9 + r];
}

/* Split a fixed-point coordinate into base voxel and fraction; returns 0 if
 * the coordinate is outside [0, (n-1)] voxels. */
static int or_split(int64_t q, int n, int *b, double *fr)
{
    if (q < 0 || q > (int64_t)(n - 1) * OR_ONE) return 0;
    int bb = (int)(q >> OR_FRAC_BITS);
    double ff = (double)(q & OR_FRAC_MASK) / (double)OR_ONE;
    if (bb == n - 1) { bb = n - 2; ff = 1.0; }
    *b = bb;
    *fr = ff;
    return 1;
}

/* Trilinear interpolation of x at fixed-point position q.  Returns 0 when
 * the position is outside the volume (then nothing is read). */
static int or_trilinear(const float *x, int nx, int ny, int nz, const int64_t q[3], double *val,
                        int b[3], double fr[3])
{
    if (!or_split(q[0], nx, &b[0], &fr[0])) return 0;
    if (!or_split(q[1], ny, &b[1], &fr[1])) return 0;
    if (!or_split(q[2], nz, &b[2], &fr[2])) return 0;
    double acc = 0.0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                double w = (cx ? fr[0] : 1.0 - fr[0]) * (cy ? fr[1] : 1.0 - fr[1])
                           * (cz ? fr[2] : 1.0 - fr[2]);
                size_t idx = ((size_t)(b[2] + cz) * ny + (size_t)(b[1] + cy)) * nx
                             + (size_t)(b[0] + cx);
                acc += w * (double)x[idx];
            }
    *val = acc;
    return 1;
}

/* Gaussian PSF weights. gxy[t + kxy], t = -kxy..kxy; gz[z + kz], z = -kz..kz. */
/* sinc(u) = sin(pi u) / (pi u) by its Maclaurin series 1 - x^2/3! + x^4/5! -
 * ..., x = pi u (Sec. II, the Taylor-series PSF): terms are added until the
 * next one is below eps times the partial sum. */
static double or_sinc_taylor(double u, double eps)
{
    double x2 = (M_PI * u) * (M_PI * u), term = 1.0, sum = 1.0;
    for (int k = 1; k < 200; ++k) {
        term *= -x2 / ((double)(2 * k) * (double)(2 * k + 1));
        sum += term;
        if (fabs(term) <= eps * fabs(sum)) break;
    }
    return sum;
}

static void or_psf_weights(const or_geom *g, const or_psf *psf, int stack, double *gxy, double *gz)
{
    double fwhm_to_sigma = 1.0 / (2.0 * sqrt(2.0 * log(2.0)));
    double sxy = psf->fwhm_xy * fwhm_to_sigma;
    double sz = g->thick[stack] * fwhm_to_sigma;
    /* sinc(u) falls to 1/2 at u = 0.6033545644..., so a sinc profile with
     * full width at half maximum F (pixels) is sinc(1.2067091288 d / F) */
    const double sinc_fwhm = 1.2067091288;
    for (int t = -psf->kxy; t <= psf->kxy; ++t) {
        if (psf->kind == 1)
            gxy[t + psf->kxy] = (psf->fwhm_xy > 0.0)
                                    ? or_sinc_taylor(sinc_fwhm * (double)t / psf->fwhm_xy, psf->eps)
                                    : (t == 0);
        else
            gxy[t + psf->kxy] = (sxy > 0.0) ? exp(-(double)(t * t) / (2.0 * sxy * sxy)) : (t == 0);
    }
    for (int z = -psf->kz; z <= psf->kz; ++z) {
        double off = (double)z * psf->dz;
        gz[z + psf->kz] = (sz > 0.0) ? exp(-(off * off) / (2.0 * sz * sz)) : (z == 0);
    }
}

void or_psf_table(const or_geom *g, const or_psf *psf, int stack, double *gxy, double *gz)
{
    or_psf_weights(g, psf, stack, gxy, gz);
}

/* ------------------------------------------------------------- simulate -- */

/* Forward model (Eq. 1 with W = D B T): every pixel of every patch is the
 * PSF-weighted mean of trilinear samples of x at the transformed sample
 * positions; samples outside the volume carry no weight.  A pixel with no
 * in-volume sample is invalid (sim = 0, valid = 0).  den (optional) receives
 * the PSF weight that fell inside the volume. */
void or_simulate(const or_geom *g, const or_psf *psf, const float *x, const int *desc,
                 const int64_t *fix, int P, double *sim, uint8_t *valid, double *den)
{
    int K = psf->kxy, Kz = psf->kz;
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p) {
        const int *d = desc + 8 * (size_t)p;
        const int64_t *f = fix + 16 * (size_t)p;
        double gxy[33], gz[65];
        or_psf_weights(g, psf, d[0], gxy, gz);
        int w = d[4], h = d[5];
        size_t off = (size_t)d[6];
        for (int j = 0; j < h; ++j)
            for (int i = 0; i < w; ++i) {
                double num = 0.0, dn = 0.0;
                if (f[12]) {
                    for (int dj = -K; dj <= K; ++dj)
                        for (int di = -K; di <= K; ++di)
                            for (int z = -Kz; z <= Kz; ++z) {
                                int64_t q[3];
                                int b[3];
                                double fr[3], v;
                                or_lattice_pos(f, i + di, j + dj, z, q);
                                if (!or_trilinear(x, g->nx, g->ny, g->nz, q, &v, b, fr)) continue;
                                double wt = gxy[di + K] * gxy[dj + K] * gz[z + Kz];
                                num += wt * v;
                                dn += wt;
                            }
                }
                size_t o = off + (size_t)j * w + i;
                valid[o] = dn > 0.0;
                sim[o] = dn > 0.0 ? num / dn : 0.0;
                if (den) den[o] = dn;
            }
    }
}

/* -------------------------------------------------------------- adjoint -- */

/* Transpose of or_simulate: addon += A^T (w .* r), conf += A^T w, where
 * A[pix][vox] = sum over the pixel's in-volume samples of (g / den) times the
 * sample's trilinear weight on vox.  w == NULL means w = 1; r == NULL means
 * r = 1.  Invalid pixels contribute nothing. */
void or_adjoint(const or_geom *g, const or_psf *psf, const int *desc, const int64_t *fix, int P,
                const double *r, const double *wgt, double *addon, double *conf)
{
    int K = psf->kxy, Kz = psf->kz;
    int nx = g->nx, ny = g->ny, nz = g->nz;
    for (int p = 0; p < P; ++p) {
        const int *d = desc + 8 * (size_t)p;
        const int64_t *f = fix + 16 * (size_t)p;
        if (!f[12]) continue;
        double gxy[33], gz[65];
        or_psf_weights(g, psf, d[0], gxy, gz);
        int w = d[4], h = d[5];
        size_t off = (size_t)d[6];
        for (int j = 0; j < h; ++j)
            for (int i = 0; i < w; ++i) {
                /* pass 1: the pixel's in-volume PSF weight */
                double dn = 0.0;
                for (int dj = -K; dj <= K; ++dj)
                    for (int di = -K; di <= K; ++di)
                        for (int z = -Kz; z <= Kz; ++z) {
                            int64_t q[3];
                            int b[3];
                            double fr[3];
                            or_lattice_pos(f, i + di, j + dj, z, q);
                            if (!or_split(q[0], nx, &b[0], &fr[0]) || !or_split(q[1], ny, &b[1], &fr[1])
                                || !or_split(q[2], nz, &b[2], &fr[2]))
                                continue;
                            dn += gxy[di + K] * gxy[dj + K] * gz[z + Kz];
                        }
                if (!(dn > 0.0)) continue;
                size_t o = off + (size_t)j * w + i;
                double wp = wgt ? wgt[o] : 1.0;
                double rp = r ? r[o] : 1.0;
                /* pass 2: scatter */
                for (int dj = -K; dj <= K; ++dj)
                    for (int di = -K; di <= K; ++di)
                        for (int z = -Kz; z <= Kz; ++z) {
                            int64_t q[3];
                            int b[3];
                            double fr[3];
                            or_lattice_pos(f, i + di, j + dj, z, q);
                            if (!or_split(q[0], nx, &b[0], &fr[0]) || !or_split(q[1], ny, &b[1], &fr[1])
                                || !or_split(q[2], nz, &b[2], &fr[2]))
                                continue;
                            double a = gxy[di + K] * gxy[dj + K] * gz[z + Kz] / dn;
                            for (int cz = 0; cz < 2; ++cz)
                                for (int cy = 0; cy < 2; ++cy)
                                    for (int cx = 0; cx < 2; ++cx) {
                                        double tw = (cx ? fr[0] : 1.0 - fr[0]) * (cy ? fr[1] : 1.0 - fr[1])
                                                    * (cz ? fr[2] : 1.0 - fr[2]);
                                        size_t idx = ((size_t)(b[2] + cz) * ny + (size_t)(b[1] + cy)) * nx
                                                     + (size_t)(b[0] + cx);
                                        if (addon) addon[idx] += wp * rp * a * tw;
                                        if (conf) conf[idx] += wp * a * tw;
                                    }
                        }
            }
    }
}

/* ----------------------------------------------------------- EM weights -- */

static double or_gauss(double e, double sigma2)
{
    return exp(-(e * e) / (2.0 * sigma2)) / (sqrt(2.0 * M_PI) * sqrt(sigma2));
}

static double or_clamp(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }


/* EM robust statistics (Sec. II "EM-Based Outlier Removal").
 *
 * 1. Residuals e = y - sim on valid pixels.  "Participating" pixels are the
 *    valid pixels of patches whose input mask is 1 (mask_in == NULL: all).
 * 2. First call (state[ST_INIT] == 0): sigma^2 = mean e^2 over the
 *    participating pixels, c = c0.
 * 3. Outlier density m = 1 / (max e - min e) over the participating pixels
 *    (Eq. for m); m = 0 when the range is below 1e-12.
 * 4. E-step on every valid pixel with the current (sigma^2, c, m):
 *    p = G_sigma(e) c / (G_sigma(e) c + m (1 - c))  (Eq. for p), p = 1 if
 *    m = 0; invalid pixels get p = 0.
 * 5. M-step over the participating pixels: sigma^2 = sum p e^2 / sum p,
 *    floored at max((sigma_floor_rel * range)^2, 1e-12); c = sum p / N,
 *    clamped to [1e-3, 1 - 1e-3].  Stored for the next call.
 * 6. Patch potential p-bar_s = sqrt(sum p^2 / N_s) over the patch's valid
 *    pixels (Eq. for p-bar).  A patch with N_s < min_valid_frac * w * h (or
 *    none) is not eligible: w_s = 0, mask 0.
 * 7. Patch classification, rule 0: the pixel-level model applied one level
 *    up.  Inlier potentials follow a one-sided Gaussian (mean mu_p, variance
 *    sigma_p^2; potentials above mu_p get the peak density), outliers a
 *    uniform density m_p = 1 / (max p-bar - min p-bar) over the eligible
 *    patches, mixing c_p.  First call: mu_p and sigma_p^2 = mean and variance
 *    of the eligible potentials (variance floored at 1e-4), c_p = c0.
 *    patch_em_iters EM iterations, warm-started from the state, then a final
 *    E-step gives w_s; mask_s = (w_s >= 0.5).  m_p = 0 gives w_s = 1.
 *    Rule 1: w_s = p-bar_s, mask_s = (p-bar_s >= patch_threshold).
 */
void or_em_weights(const float *y, const double *sim, const uint8_t *valid, const int *desc, int P,
                   const or_em_params *ep, double *state, const uint8_t *mask_in,
                   uint8_t *mask_out, double *p_out, double *w_patch, double *pbar)
{
    /* 1-3 */
    double emin = INFINITY, emax = -INFINITY, se2 = 0.0, npart = 0.0;
    for (int s = 0; s < P; ++s) {
        const int *d = desc + 8 * (size_t)s;
        if (mask_in && !mask_in[s]) continue;
        size_t off = (size_t)d[6], n = (size_t)d[4] * (size_t)d[5];
        for (size_t t = 0; t < n; ++t) {
            if (!valid[off + t]) continue;
            double e = (double)y[off + t] - sim[off + t];
            emin = e < emin ? e : emin;
            emax = e > emax ? e : emax;
            se2 += e * e;
            npart += 1.0;
        }
    }
    double range = (npart > 0.0) ? emax - emin : 0.0;
    double sfloor = (ep->sigma_floor_rel * range) * (ep->sigma_floor_rel * range);
    if (sfloor < 1e-12) sfloor = 1e-12;
    int first = state[ST_INIT] == 0.0;
    if (first) {
        double s2 = npart > 0.0 ? se2 / npart : 1.0;
        state[ST_SIGMA2] = s2 < sfloor ? sfloor : s2;
        state[ST_C] = or_clamp(ep->c0, 1e-3, 1.0 - 1e-3);
    }
    double m = (range >= 1e-12) ? 1.0 / range : 0.0;
    double sigma2 = state[ST_SIGMA2], c = state[ST_C];

    /* 4 */
    for (int s = 0; s < P; ++s) {
        const int *d = desc + 8 * (size_t)s;
        size_t off = (size_t)d[6], n = (size_t)d[4] * (size_t)d[5];
        for (size_t t = 0; t < n; ++t) {
            double pv = 0.0;
            if (valid[off + t]) {
                if (m == 0.0) {
                    pv = 1.0;
                } else {
                    double e = (double)y[off + t] - sim[off + t];
                    double G = or_gauss(e, sigma2);
                    pv = (G * c) / (G * c + m * (1.0 - c));
                }
            }
            p_out[off + t] = pv;
        }
    }

    /* 5 */
    double sp = 0.0, spe2 = 0.0;
    for (int s = 0; s < P; ++s) {
        const int *d = desc + 8 * (size_t)s;
        if (mask_in && !mask_in[s]) continue;
        size_t off = (size_t)d[6], n = (size_t)d[4] * (size_t)d[5];
        for (size_t t = 0; t < n; ++t) {
            if (!valid[off + t]) continue;
            double e = (double)y[off + t] - sim[off + t];
            sp += p_out[off + t];
            spe2 += p_out[off + t] * e * e;
        }
    }
    if (sp > 0.0) {
        double s2 = spe2 / sp;
        state[ST_SIGMA2] = s2 < sfloor ? sfloor : s2;
    }
    if (npart > 0.0) state[ST_C] = or_clamp(sp / npart, 1e-3, 1.0 - 1e-3);

    /* 6 */
    uint8_t *elig = (uint8_t *)calloc((size_t)(P > 0 ? P : 1), 1);
    double pmin = INFINITY, pmax = -INFINITY, psum = 0.0, nelig = 0.0;
    for (int s = 0; s < P; ++s) {
        const int *d = desc + 8 * (size_t)s;
        size_t off = (size_t)d[6], n = (size_t)d[4] * (size_t)d[5];
        double sp2 = 0.0, nv = 0.0;
        for (size_t t = 0; t < n; ++t)
            if (valid[off + t]) {
                sp2 += p_out[off + t] * p_out[off + t];
                nv += 1.0;
            }
        pbar[s] = nv > 0.0 ? sqrt(sp2 / nv) : 0.0;
        elig[s] = nv > 0.0 && nv >= ep->min_valid_frac * (double)n;
        if (elig[s]) {
            pmin = pbar[s] < pmin ? pbar[s] : pmin;
            pmax = pbar[s] > pmax ? pbar[s] : pmax;
            psum += pbar[s];
            nelig += 1.0;
        }
    }

    /* 7 */
    if (ep->patch_rule == 1) {
        for (int s = 0; s < P; ++s) {
            w_patch[s] = elig[s] ? pbar[s] : 0.0;
            mask_out[s] = elig[s] && pbar[s] >= ep->patch_threshold;
        }
    } else {
        double mp = (nelig > 0.0 && pmax - pmin >= 1e-12) ? 1.0 / (pmax - pmin) : 0.0;
        if (first) {
            double mu = nelig > 0.0 ? psum / nelig : 0.0, var = 0.0;
            for (int s = 0; s < P; ++s)
                if (elig[s]) var += (pbar[s] - mu) * (pbar[s] - mu);
            var = nelig > 0.0 ? var / nelig : 0.0;
            state[ST_MU_P] = mu;
            state[ST_SIGMA2_P] = var < 1e-4 ? 1e-4 : var;
            state[ST_C_P] = or_clamp(ep->c0, 1e-3, 1.0 - 1e-3);
        }
        for (int it = 0; it <= ep->patch_em_iters; ++it) {
            double mu = state[ST_MU_P], v2 = state[ST_SIGMA2_P], cp = state[ST_C_P];
            for (int s = 0; s < P; ++s) {
                if (!elig[s]) { w_patch[s] = 0.0; continue; }
                if (mp == 0.0) { w_patch[s] = 1.0; continue; }
                double dlt = pbar[s] >= mu ? 0.0 : pbar[s] - mu;
                double G = or_gauss(dlt, v2);
                w_patch[s] = (G * cp) / (G * cp + mp * (1.0 - cp));
            }
            if (it == ep->patch_em_iters || mp == 0.0) break;
            double sw = 0.0, swp = 0.0;
            for (int s = 0; s < P; ++s)
                if (elig[s]) { sw += w_patch[s]; swp += w_patch[s] * pbar[s]; }
            if (!(sw > 0.0)) break;
            double mu_n = swp / sw, swv = 0.0;
            for (int s = 0; s < P; ++s)
                if (elig[s]) swv += w_patch[s] * ((pbar[s] - mu_n) * (pbar[s] - mu_n));
            double v2n = swv / sw;
            state[ST_MU_P] = mu_n;
            state[ST_SIGMA2_P] = v2n < 1e-4 ? 1e-4 : v2n;
            state[ST_C_P] = or_clamp(sw / nelig, 1e-3, 1.0 - 1e-3);
        }
        state[ST_M_P] = mp;
        for (int s = 0; s < P; ++s) mask_out[s] = elig[s] && w_patch[s] >= 0.5;
    }
    double nin = 0.0;
    for (int s = 0; s < P; ++s) nin += mask_out[s];
    free(elig);

    state[ST_INIT] = 1.0;
    state[ST_SIGMA2_USED] = sigma2;
    state[ST_M] = m;
    state[ST_EMIN] = emin;
    state[ST_EMAX] = emax;
    state[ST_N_PART] = npart;
    state[ST_SUM_P] = sp;
    state[ST_SUM_PE2] = spe2;
    state[ST_N_ELIG] = nelig;
    state[ST_N_IN] = nin;
}

/* -------------------------------------------------------- volume update -- */

/* Weighted SIRT step of the super-resolution update: rows of A sum to one,
 * so x += alpha * A^T(w e) / A^T(w) wherever A^T(w) > conf_eps, then x is
 * clamped at zero.  Voxels no sample reached keep their value. */
void or_volume_update(double *x, const double *addon, const double *conf, size_t n, double alpha,
                      double conf_eps)
{
    for (size_t v = 0; v < n; ++v) {
        if (conf[v] > conf_eps) {
            double nv = x[v] + alpha * addon[v] / conf[v];
            x[v] = nv > 0.0 ? nv : 0.0;
        }
    }
}

/* Regularised super-resolution update (reading of the edge-preserving
 * regularisation by anisotropic diffusion of the SR framework PVR builds
 * on; the paper prints no formula).  First the SIRT step of
 * or_volume_update gives u.  Then every voxel v reached by the data
 * (conf > conf_eps) takes one explicit diffusion step over its 26
 * neighbours d inside the volume:
 *   x(v) = max(u(v) + lambda * sum_d w_d psi(u(v + d) - u(v)), 0),
 *   psi(D) = D / sqrt(1 + (D / delta)^2)   (edge-stopping flux: about D for
 *            differences well below delta, bounded by delta above it),
 *   w_d = (1 / |d|^2) / W,  W = 6 + 12 / 2 + 8 / 3 = 44 / 3,
 * |d| in voxel steps, so the weights of a full neighbourhood sum to one and
 * 0 <= lambda <= 1 keeps the step a convex combination for small
 * differences.  Voxels the data did not reach keep u.  x: [nz][ny][nx]. */
void or_sr_update(double *x, const double *addon, const double *conf, int nx, int ny, int nz, double alpha,
                  double conf_eps, double lambda, double delta)
{
    size_t n = (size_t)nx * ny * nz;
    double *u = (double *)malloc(n * sizeof(double));
    memcpy(u, x, n * sizeof(double));
    or_volume_update(u, addon, conf, n, alpha, conf_eps);
    const double W = 6.0 + 12.0 / 2.0 + 8.0 / 3.0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int xx = 0; xx < nx; ++xx) {
                size_t v = ((size_t)z * ny + y) * nx + xx;
                if (!(conf[v] > conf_eps)) {
                    x[v] = u[v];
                    continue;
                }
                double flux = 0.0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 == 0) continue;
                            int qx = xx + dx, qy = y + dy, qz = z + dz;
                            if (qx < 0 || qy < 0 || qz < 0 || qx >= nx || qy >= ny || qz >= nz) continue;
                            double D = u[((size_t)qz * ny + qy) * nx + qx] - u[v];
                            double psi = D / sqrt(1.0 + (D / delta) * (D / delta));
                            flux += (1.0 / (double)r2) / W * psi;
                        }
                double nv = u[v] + lambda * flux;
                x[v] = nv > 0.0 ? nv : 0.0;
            }
    free(u);
}

/* -------------------------------------------------------- registration -- */

/* Derivatives of the linear part of the transform with respect to each pose
 * parameter (3x3 each, dL[k - 3] for k = 3..n_params-1).  Rigid: d(Rz Ry
 * Rx)/d angle per degree (libm trigonometry: the gradient is not part of
 * the bit-exact integer path); affine: the unit matrix E_rc. */
static void or_dlinear(const double *th, int n_params, double dL[9][9])
{
    if (n_params == 12) {
        for (int k = 0; k < 9; ++k) {
            memset(dL[k], 0, 9 * sizeof(double));
            dL[k][k] = 1.0;
        }
        return;
    }
    double ax = th[3] * M_PI / 180.0, ay = th[4] * M_PI / 180.0, az = th[5] * M_PI / 180.0;
    double Rx[9] = {1, 0, 0, 0, cos(ax), -sin(ax), 0, sin(ax), cos(ax)};
    double Ry[9] = {cos(ay), 0, sin(ay), 0, 1, 0, -sin(ay), 0, cos(ay)};
    double Rz[9] = {cos(az), -sin(az), 0, sin(az), cos(az), 0, 0, 0, 1};
    double dRx[9] = {0, 0, 0, 0, -sin(ax), -cos(ax), 0, cos(ax), -sin(ax)};
    double dRy[9] = {-sin(ay), 0, cos(ay), 0, 0, 0, -cos(ay), 0, -sin(ay)};
    double dRz[9] = {-sin(az), -cos(az), 0, cos(az), -sin(az), 0, 0, 0, 0};
    for (int k = 3; k < 6; ++k) {
        const double *A = (k == 5) ? dRz : Rz;
        const double *B = (k == 4) ? dRy : Ry;
        const double *Cm = (k == 3) ? dRx : Rx;
        double AB[9];
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) {
                AB[r * 3 + cc] = 0.0;
                for (int t = 0; t < 3; ++t) AB[r * 3 + cc] += A[r * 3 + t] * B[t * 3 + cc];
            }
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) {
                double v = 0.0;
                for (int t = 0; t < 3; ++t) v += AB[r * 3 + t] * Cm[t * 3 + cc];
                dL[k - 3][r * 3 + cc] = v * (M_PI / 180.0);
            }
    }
}

/* Derivative of the transformed world point T(w) = L (w - c) + c + t with
 * respect to pose parameter k at world point w (before the transform). */
static void or_dT_dtheta(const double dL[9][9], int k, const double c[3], const double w[3],
                         double out[3])
{
    double u[3] = {w[0] - c[0], w[1] - c[1], w[2] - c[2]};
    memset(out, 0, 3 * sizeof(double));
    if (k < 3) { out[k] = 1.0; return; }
    const double *D = dL[k - 3];
    for (int r = 0; r < 3; ++r) out[r] = D[r * 3 + 0] * u[0] + D[r * 3 + 1] * u[1] + D[r * 3 + 2] * u[2];
}

/* Sample position for the registration evaluation.  With exact = 1 the
 * fixed-point lattice is used (what the method computes); with exact = 0 the
 * position is taken in plain FP64 from the pose matrix, which is smooth in
 * the pose and serves the finite-difference checks of the gradient. */
static int or_reg_sample(const or_geom *g, const float *x, const int64_t *f, const double *M,
                         double zs, const int *d, int exact, int i, int j, int z, double *val,
                         double grad[3])
{
    int nx = g->nx, ny = g->ny, nz = g->nz;
    int n[3] = {nx, ny, nz};
    int b[3];
    double fr[3];
    if (exact) {
        int64_t q[3];
        or_lattice_pos(f, i, j, z, q);
        for (int r = 0; r < 3; ++r)
            if (!or_split(q[r], n[r], &b[r], &fr[r])) return 0;
    } else {
        double px = (double)(d[2] + i), py = (double)(d[3] + j), pk = (double)d[1] + (double)z * zs;
        for (int r = 0; r < 3; ++r) {
            double qc = M[r * 4 + 0] * px + M[r * 4 + 1] * py + M[r * 4 + 2] * pk + M[r * 4 + 3];
            if (qc < 0.0 || qc > (double)(n[r] - 1)) return 0;
            double fl = floor(qc);
            b[r] = (int)fl;
            fr[r] = qc - fl;
            if (b[r] == n[r] - 1) { b[r] = n[r] - 2; fr[r] = 1.0; }
        }
    }
    double v = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                double wx = cx ? fr[0] : 1.0 - fr[0], wy = cy ? fr[1] : 1.0 - fr[1];
                double wz = cz ? fr[2] : 1.0 - fr[2];
                double sx = cx ? 1.0 : -1.0, sy = cy ? 1.0 : -1.0, sz = cz ? 1.0 : -1.0;
                double xv = (double)x[((size_t)(b[2] + cz) * ny + (size_t)(b[1] + cy)) * nx
                                      + (size_t)(b[0] + cx)];
                v += wx * wy * wz * xv;
                gx += sx * wy * wz * xv;
                gy += wx * sy * wz * xv;
                gz += wx * wy * sz * xv;
            }
    *val = v;
    grad[0] = gx;
    grad[1] = gy;
    grad[2] = gz;
    return 1;
}

/* Simulated value s, validity ok and pose Jacobian J = d s / d theta
 * (n_params per pixel) of every pixel of one patch at pose th, by the
 * definition of the forward model (Eq. 1: PSF-weighted trilinear samples
 * over the in-volume PSF weight) differentiated through the sample
 * positions: d s / d theta = sum_samples g * grad_trilinear . d q / d theta
 * / den, the normalisation den treated as constant (it changes only where a
 * sample leaves the volume).  exact selects the fixed-point lattice or plain
 * FP64 positions (or_reg_sample).  member (indexed like the patch pixels,
 * may be NULL): pixels with member 0 are not part of the patch.  Returns 0
 * when the exact lattice is out of range (every pixel invalid). */
static int or_patch_sim_jac(const or_geom *g, const or_psf *psf, const float *x, const int *d,
                            const double *th, int n_params, int exact, const uint8_t *member,
                            double *s, uint8_t *ok, double *J)
{
    int K = psf->kxy, Kz = psf->kz, w = d[4], h = d[5];
    int64_t f[16];
    double M[12], gxy[33], gzt[65], c[3];
    or_pose_fixed(g, psf, d, th, n_params, f);
    or_patch_matrix(g, d, th, n_params, M);
    double zs = or_zeta_scale(g, d[0], psf->dz);
    or_psf_weights(g, psf, d[0], gxy, gzt);
    or_patch_centre(g, d, c);
    const double *S = g->p2w[d[0]];
    const double *W = g->w2v;
    double dL[9][9];
    or_dlinear(th, n_params, dL);
    if (exact && !f[12]) return 0;
    for (int j = 0; j < h; ++j)
        for (int i = 0; i < w; ++i) {
            double num = 0.0, dn = 0.0, jac[12] = {0};
            for (int dj = -K; dj <= K; ++dj)
                for (int di = -K; di <= K; ++di)
                    for (int z = -Kz; z <= Kz; ++z) {
                        double v, gr[3];
                        if (!or_reg_sample(g, x, f, M, zs, d, exact, i + di, j + dj, z, &v, gr)) continue;
                        double wt = gxy[di + K] * gxy[dj + K] * gzt[z + Kz];
                        num += wt * v;
                        dn += wt;
                        /* world point of the sample before the transform */
                        double px = (double)(d[2] + i + di), py = (double)(d[3] + j + dj);
                        double pk = (double)d[1] + (double)z * zs, wp[3];
                        for (int r = 0; r < 3; ++r)
                            wp[r] = S[r * 4 + 0] * px + S[r * 4 + 1] * py + S[r * 4 + 2] * pk + S[r * 4 + 3];
                        for (int k = 0; k < n_params; ++k) {
                            double dT[3], dq[3];
                            or_dT_dtheta(dL, k, c, wp, dT);
                            for (int r = 0; r < 3; ++r)
                                dq[r] = W[r * 4 + 0] * dT[0] + W[r * 4 + 1] * dT[1] + W[r * 4 + 2] * dT[2];
                            jac[k] += wt * (gr[0] * dq[0] + gr[1] * dq[1] + gr[2] * dq[2]);
                        }
                    }
            size_t o = (size_t)j * w + i;
            if (dn > 0.0 && (!member || member[(size_t)d[6] + o])) {
                ok[o] = 1;
                s[o] = num / dn;
                for (int k = 0; k < n_params; ++k) J[o * n_params + k] = jac[k] / dn;
            }
        }
    return 1;
}

/* Pose gradient of sum_pix r_pix s_pix for one patch (the vector-Jacobian
 * product of the forward model with respect to the patch pose, what the
 * backward pass of a differentiable simulate needs), with r indexed like
 * the patch pixels (offset d[6]).  Returns sum_pix r_pix s_pix over the
 * valid pixels; grad receives n_params values. */
double or_sim_pose_vjp(const or_geom *g, const or_psf *psf, const float *x, const double *r,
                       const int *d, const double *th, int n_params, int exact, const uint8_t *member,
                       double *grad)
{
    size_t npx = (size_t)d[4] * d[5], off = (size_t)d[6];
    for (int k = 0; k < n_params; ++k) grad[k] = 0.0;
    double *s = (double *)calloc(npx, sizeof(double));
    double *J = (double *)calloc(npx * (size_t)n_params, sizeof(double));
    uint8_t *ok = (uint8_t *)calloc(npx, 1);
    double val = 0.0;
    if (or_patch_sim_jac(g, psf, x, d, th, n_params, exact, member, s, ok, J))
        for (size_t o = 0; o < npx; ++o)
            if (ok[o]) {
                val += r[off + o] * s[o];
                for (int k = 0; k < n_params; ++k) grad[k] += r[off + o] * J[o * n_params + k];
            }
    free(s);
    free(J);
    free(ok);
    return val;
}

/* NCC between the acquired patch y and the patch simulated at pose th, and
 * its gradient with respect to the pose (Sec. II: registration maximises CC,
 * Eq. cross_corr with population standard deviations, over valid pixels).
 * d sim / d theta = sum_samples g * grad_trilinear . d q / d theta / den, the
 * normalisation den being treated as constant.  Fewer than min_valid valid
 * pixels or a (near-)constant patch give NCC = 0 and a zero gradient.
 * Returns the NCC; grad receives n_params values. */
double or_ncc_grad(const or_geom *g, const or_psf *psf, const float *x, const float *y,
                   const int *d, const double *th, int n_params, int min_valid, int exact,
                   const uint8_t *member, double *grad)
{
    size_t npx = (size_t)d[4] * d[5], off = (size_t)d[6];
    for (int k = 0; k < n_params; ++k) grad[k] = 0.0;
    double *s = (double *)calloc(npx, sizeof(double));
    double *J = (double *)calloc(npx * (size_t)n_params, sizeof(double));
    uint8_t *ok = (uint8_t *)calloc(npx, 1);
    if (!or_patch_sim_jac(g, psf, x, d, th, n_params, exact, member, s, ok, J)) {
        free(s);
        free(J);
        free(ok);
        return 0.0;
    }
    double n = 0.0, my = 0.0, ms = 0.0;
    for (size_t o = 0; o < npx; ++o)
        if (ok[o]) { n += 1.0; my += y[off + o]; ms += s[o]; }
    double ncc = 0.0;
    if (n >= (double)min_valid && n > 0.0) {
        my /= n;
        ms /= n;
        double vy = 0.0, vs = 0.0, cv = 0.0;
        for (size_t o = 0; o < npx; ++o)
            if (ok[o]) {
                double a = y[off + o] - my, b = s[o] - ms;
                vy += a * a;
                vs += b * b;
                cv += a * b;
            }
        vy /= n;
        vs /= n;
        cv /= n;
        if (vy > 1e-12 * (my * my + 1.0) && vs > 1e-12 * (ms * ms + 1.0)) {
            double sd = sqrt(vy * vs);
            ncc = cv / sd;
            for (size_t o = 0; o < npx; ++o)
                if (ok[o]) {
                    double dnds = ((y[off + o] - my) / sd - ncc * (s[o] - ms) / vs) / n;
                    for (int k = 0; k < n_params; ++k) grad[k] += dnds * J[o * n_params + k];
                }
        }
    }
    free(s);
    free(J);
    free(ok);
    return ncc;
}

/* Patch-wise gradient ascent on NCC (Sec. II registration; Sec. III "patch-
 * wise gradient descent").  Per patch, n_eval NCC evaluations: the first at
 * the current pose, each later one at best + delta * g / |g| (g the gradient
 * at the best pose so far).  A trial that strictly improves NCC becomes the
 * best pose; otherwise delta is halved.  The patch stops when delta drops
 * below delta_min, the gradient vanishes or NCC is degenerate.  In fixed-step
 * mode every trial is accepted and delta stays delta0.  Steps are taken in
 * scaled parameters so that one unit moves the patch edge by about 1 mm:
 * translations in mm, rigid angles times the patch half-diagonal r (mm) in
 * radians, affine entries times r.  After an accepted trial delta is
 * multiplied by grow (1 = plain halving scheme).
 * poses are updated in place; ncc_out receives the best NCC.  margin_out
 * (may be NULL) receives per patch the smallest |NCC(trial) - NCC(best)|
 * over the acceptance decisions taken (infinity if none): a test that
 * compares another implementation's accept / reject path with this one can
 * tell which decisions lie within rounding of a tie. */
void or_register(const or_geom *g, const or_psf *psf, const or_reg_params *rp, const float *x,
                 const float *y, const int *desc, int P, double *poses, double *ncc_out,
                 double *margin_out)
{
    int np = rp->n_params;
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p) {
        const int *d = desc + 8 * (size_t)p;
        double *th = poses + (size_t)np * p;
        double best[12], gbest[12], trial[12], gt[12], scale[12];
        double half_diag = 1.0;
        {
            const double *S = g->p2w[d[0]];
            double cw = sqrt(S[0] * S[0] + S[4] * S[4] + S[8] * S[8]) * (double)d[4];
            double ch = sqrt(S[1] * S[1] + S[5] * S[5] + S[9] * S[9]) * (double)d[5];
            half_diag = 0.5 * sqrt(cw * cw + ch * ch);
        }
        for (int k = 0; k < np; ++k)
            scale[k] = k < 3 ? 1.0 : (np == 12 ? half_diag : half_diag * (M_PI / 180.0));
        memcpy(best, th, sizeof(double) * np);
        double nbest = or_ncc_grad(g, psf, x, y, d, best, np, rp->min_valid, 1, NULL, gbest);
        double delta = rp->delta0;
        double margin = INFINITY;
        int done = (nbest == 0.0);
        for (int ev = 1; ev < rp->n_eval && !done; ++ev) {
            /* step in scaled coordinates u = theta * scale: du = delta * gu / |gu|,
             * gu = g / scale */
            double gn = 0.0;
            for (int k = 0; k < np; ++k) gn += (gbest[k] / scale[k]) * (gbest[k] / scale[k]);
            gn = sqrt(gn);
            if (!(gn > 0.0)) break;
            for (int k = 0; k < np; ++k) trial[k] = best[k] + delta * (gbest[k] / scale[k]) / gn / scale[k];
            double nt = or_ncc_grad(g, psf, x, y, d, trial, np, rp->min_valid, 1, NULL, gt);
            if (fabs(nt - nbest) < margin) margin = fabs(nt - nbest);
            if (rp->fixed_step || nt > nbest) {
                memcpy(best, trial, sizeof(double) * np);
                memcpy(gbest, gt, sizeof(double) * np);
                nbest = nt;
                if (!rp->fixed_step) delta *= rp->grow;
            } else {
                delta *= 0.5;
                if (delta < rp->delta_min) done = 1;
            }
        }
        memcpy(th, best, sizeof(double) * np);
        if (ncc_out) ncc_out[p] = nbest;
        if (margin_out) margin_out[p] = margin;
    }
}

/* ---------------------------------------------------------------- metrics -- */

/* Evaluation metrics of Sec. IV-A over n values (mask == NULL: all):
 * m[0] PSNR = 10 log10(I_max^2 / MSE), I_max = max of the reference (Eq. PSNR,
 *      logarithm read as base 10);
 * m[1] CC = mean of the product of standardised values, population standard
 *      deviations (Eq. cross_corr);
 * m[2] SSIM, single global window, with the denominator's first factor read
 *      as mu_I^2 + mu_J^2 + c1 (Eq. SSIM), c1 = (0.01 L)^2, c2 = (0.03 L)^2,
 *      L = max - min of the reference;
 * m[3] DSSIM = (1 - SSIM) / 2 (Eq. DSSIM);
 * m[4] MSE. */
void or_metrics(const double *ref, const double *img, const uint8_t *mask, size_t n, double *mo)
{
    double cnt = 0.0, mr = 0.0, mi = 0.0, rmax = -INFINITY, rmin = INFINITY;
    for (size_t t = 0; t < n; ++t) {
        if (mask && !mask[t]) continue;
        cnt += 1.0;
        mr += ref[t];
        mi += img[t];
        rmax = ref[t] > rmax ? ref[t] : rmax;
        rmin = ref[t] < rmin ? ref[t] : rmin;
    }
    for (int k = 0; k < 5; ++k) mo[k] = 0.0;
    if (cnt == 0.0) return;
    mr /= cnt;
    mi /= cnt;
    double vr = 0.0, vi = 0.0, cv = 0.0, se = 0.0;
    for (size_t t = 0; t < n; ++t) {
        if (mask && !mask[t]) continue;
        double a = ref[t] - mr, b = img[t] - mi, dd = img[t] - ref[t];
        vr += a * a;
        vi += b * b;
        cv += a * b;
        se += dd * dd;
    }
    vr /= cnt;
    vi /= cnt;
    cv /= cnt;
    double mse = se / cnt;
    mo[0] = mse > 0.0 ? 10.0 * log10(rmax * rmax / mse) : INFINITY;
    mo[1] = (vr > 0.0 && vi > 0.0) ? cv / sqrt(vr * vi) : 0.0;
    double L = rmax - rmin, c1 = (0.01 * L) * (0.01 * L), c2 = (0.03 * L) * (0.03 * L);
    double ssim = ((2.0 * mr * mi + c1) * (2.0 * cv + c2)) / ((mr * mr + mi * mi + c1) * (vr + vi + c2));
    mo[2] = ssim;
    mo[3] = (1.0 - ssim) / 2.0;
    mo[4] = mse;
}

/* ---------------------------------------------------------- patch table -- */

/* Per-patch evaluation (Sec. IV-A: metrics between the acquired patches and
 * the patches simulated from the reconstruction).  For every patch, over its
 * valid pixels: out[5p..5p+4] = {PSNR, CC, SSIM, DSSIM} of or_metrics with
 * the acquired patch as reference, and the mean of the local SSIM map.  The
 * DSSIM heat map (Eq. DSSIM, visualised as maps in Sec. V) takes SSIM over
 * the valid pixels of the (2w+1) x (2w+1) window around each pixel, clipped
 * to the patch, with the patch's c1, c2 (L = range of the acquired patch):
 * map[pix] = (1 - SSIM_local) / 2, 0 at invalid pixels. */
void or_patch_metrics(const float *y, const float *sim, const uint8_t *valid, const int *desc,
                      int P, int w, double *out, double *map)
{
    for (int p = 0; p < P; ++p) {
        const int *d = desc + 8 * (size_t)p;
        int W = d[4], H = d[5];
        size_t off = (size_t)d[6], n = (size_t)W * H;
        double *ref = (double *)malloc(n * sizeof(double)), *img = (double *)malloc(n * sizeof(double));
        for (size_t t = 0; t < n; ++t) {
            ref[t] = y[off + t];
            img[t] = sim[off + t];
        }
        double mo[5];
        or_metrics(ref, img, valid + off, n, mo);
        double rmax = -INFINITY, rmin = INFINITY;
        for (size_t t = 0; t < n; ++t)
            if (valid[off + t]) {
                rmax = ref[t] > rmax ? ref[t] : rmax;
                rmin = ref[t] < rmin ? ref[t] : rmin;
            }
        double L = rmax - rmin, c1 = (0.01 * L) * (0.01 * L), c2 = (0.03 * L) * (0.03 * L);
        double ssum = 0.0, scnt = 0.0;
        for (int j = 0; j < H; ++j)
            for (int i = 0; i < W; ++i) {
                size_t t = (size_t)j * W + i;
                map[off + t] = 0.0;
                if (!valid[off + t]) continue;
                double k = 0.0, ma = 0.0, mb = 0.0;
                for (int jj = j - w; jj <= j + w; ++jj)
                    for (int ii = i - w; ii <= i + w; ++ii) {
                        if (ii < 0 || jj < 0 || ii >= W || jj >= H) continue;
                        size_t u = (size_t)jj * W + ii;
                        if (!valid[off + u]) continue;
                        k += 1.0;
                        ma += ref[u];
                        mb += img[u];
                    }
                ma /= k;
                mb /= k;
                double va = 0.0, vb = 0.0, cab = 0.0;
                for (int jj = j - w; jj <= j + w; ++jj)
                    for (int ii = i - w; ii <= i + w; ++ii) {
                        if (ii < 0 || jj < 0 || ii >= W || jj >= H) continue;
                        size_t u = (size_t)jj * W + ii;
                        if (!valid[off + u]) continue;
                        va += (ref[u] - ma) * (ref[u] - ma);
                        vb += (img[u] - mb) * (img[u] - mb);
                        cab += (ref[u] - ma) * (img[u] - mb);
                    }
                va /= k;
                vb /= k;
                cab /= k;
                double ss = ((2.0 * ma * mb + c1) * (2.0 * cab + c2)) / ((ma * ma + mb * mb + c1) * (va + vb + c2));
                map[off + t] = (1.0 - ss) / 2.0;
                ssum += ss;
                scnt += 1.0;
            }
        for (int k = 0; k < 4; ++k) out[5 * (size_t)p + k] = mo[k];
        out[5 * (size_t)p + 4] = scnt > 0.0 ? ssum / scnt : 0.0;
        free(ref);
        free(img);
    }
}

/* Square patches of side a and stride stride on every slice of every stack
 * (Sec. II "Patch Extraction"): corners x0, y0 = 0, stride, 2 stride, ...
 * while x0 + a <= W (resp. y0 + a <= H), in the order stack, slice, y0, x0.
 * A patch is kept when at least keep_frac * a^2 of its pixels exceed the
 * foreground level fg_frac * I_max, I_max the largest pixel of all stacks;
 * the level and the comparison are taken in single precision, the count
 * test in double.  desc rows: {stack, slice, x0, y0, a, a, pix_off, 0}.
 * Returns the number of patches (at most max_out rows are written);
 * *npix receives the total pixel count of the kept patches.
 * or_patches_build_sizes takes the side a and stride of every slice from
 * slice_a[] and slice_stride[] (slices numbered over all stacks in order):
 * patches of several scales (Sec. II builds its patch sets at several
 * sizes); or_patches_build is the single-size case. */
int or_patches_build_sizes(const or_geom *g, const float *stacks, const int *slice_a,
                           const int *slice_stride, double fg_frac, double keep_frac, int *desc,
                           int max_out, int64_t *npix)
{
    size_t total = 0;
    for (int s = 0; s < g->n_stacks; ++s) total += (size_t)g->sw[s] * g->sh[s] * g->sk[s];
    float imax = -INFINITY;
    for (size_t t = 0; t < total; ++t) imax = stacks[t] > imax ? stacks[t] : imax;
    float thr = (float)fg_frac * imax;
    int n = 0;
    int64_t off = 0;
    size_t soff = 0;
    int gk = 0;   /* slice index over all stacks */
    for (int s = 0; s < g->n_stacks; ++s) {
        int W = g->sw[s], H = g->sh[s], Kk = g->sk[s];
        for (int k = 0; k < Kk; ++k, ++gk) {
            int a = slice_a[gk], stride = slice_stride[gk];
            for (int y0 = 0; y0 + a <= H; y0 += stride)
                for (int x0 = 0; x0 + a <= W; x0 += stride) {
                    long cnt = 0;
                    for (int j = 0; j < a; ++j)
                        for (int i = 0; i < a; ++i)
                            cnt += stacks[soff + ((size_t)k * H + (y0 + j)) * W + (x0 + i)] > thr;
                    if (!((double)cnt >= keep_frac * (double)a * (double)a)) continue;
                    if (n < max_out) {
                        int *d = desc + 8 * (size_t)n;
                        d[0] = s; d[1] = k; d[2] = x0; d[3] = y0; d[4] = a; d[5] = a;
                        d[6] = (int)off; d[7] = 0;
                    }
                    off += (int64_t)a * a;
                    ++n;
                }
        }
        soff += (size_t)W * H * Kk;
    }
    *npix = off;
    return n;
}

int or_patches_build(const or_geom *g, const float *stacks, int a, int stride, double fg_frac,
                     double keep_frac, int *desc, int max_out, int64_t *npix)
{
    int nk = 0;
    for (int s = 0; s < g->n_stacks; ++s) nk += g->sk[s];
    int *sa = (int *)malloc((size_t)(nk > 0 ? nk : 1) * sizeof(int));
    int *ss = (int *)malloc((size_t)(nk > 0 ? nk : 1) * sizeof(int));
    for (int i = 0; i < nk; ++i) { sa[i] = a; ss[i] = stride; }
    int n = or_patches_build_sizes(g, stacks, sa, ss, fg_frac, keep_frac, desc, max_out, npix);
    free(sa);
    free(ss);
    return n;
}
