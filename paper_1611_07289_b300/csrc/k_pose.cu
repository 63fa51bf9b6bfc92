// K1: patch pose -> fixed-point sample lattice (Eq. 1: the motion part T_i
// of W_i = D B T_i), one thread per patch, float64.  Rigid poses (6
// parameters: translation in mm, Rz Ry Rx angles in degrees) or affine poses
// (12: translation and the 3x3 matrix D of the linear part I + D, row-major).
//
// The integer lattice must be reproducible bit for bit by any IEEE machine,
// so every float64 operation is an explicit round-to-nearest intrinsic
// (never contracted into an FMA), evaluated in a fixed order, and the sine
// and cosine come from their Maclaurin series after reduction to +-45
// degrees instead of the math library.
#include "pvr_internal.h"

namespace pvr {
namespace {

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// One nesting step N of the sine and cosine series and the steps below it:
// ts <- 1 - x^2 ts / ((2N)(2N+1)), tc <- 1 - x^2 tc / ((2N-1)(2N)), each
// division a multiplication by the correctly rounded reciprocal of the
// integer denominator (a compile-time IEEE double constant).
template <int N>
__device__ __forceinline__ void series_steps(double x2, double &ts, double &tc)
{
    constexpr double is = 1.0 / (double)((2 * N) * (2 * N + 1));
    constexpr double ic = 1.0 / (double)((2 * N - 1) * (2 * N));
    ts = dsub(1.0, dmul(dmul(x2, ts), is));
    tc = dsub(1.0, dmul(dmul(x2, tc), ic));
    if constexpr (N > 1) series_steps<N - 1>(x2, ts, tc);
}

// sin, cos of an angle in degrees: nearest multiple k of 90 degrees, rest
// r in [-45, 45] degrees, x = r * pi/180, then sin x = x (1 - x^2/(2*3) (1 -
// x^2/(4*5) (...))) and cos x = 1 - x^2/(1*2) (1 - x^2/(3*4) (...)) with 11
// nested factors each (truncation error < 1e-26 for |x| <= pi/4), every
// factor a multiplication by the correctly rounded reciprocal of its
// denominator (float64 division is a long instruction sequence); the
// quadrant k mod 4 permutes and negates the pair.
__device__ void sincos_deg_series(double deg, double *s_out, double *c_out)
{
    double k = rint(ddiv(deg, 90.0));
    double r = dsub(deg, dmul(90.0, k));
    double x = dmul(r, 0.017453292519943295769);
    double x2 = dmul(x, x);
    double ts = 1.0, tc = 1.0;
    series_steps<11>(x2, ts, tc);
    double sr = dmul(x, ts), cr = tc;
    long long q = ((long long)fmod(k, 4.0) + 4) % 4;
    if (q == 0) { *s_out = sr; *c_out = cr; }
    else if (q == 1) { *s_out = cr; *c_out = -sr; }
    else if (q == 2) { *s_out = -sr; *c_out = -cr; }
    else { *s_out = -cr; *c_out = sr; }
}

// R = Rz(rz) Ry(ry) Rx(rx), closed-form entries.
__device__ void rotation_zyx(const double *th, double L[9])
{
    double sx, cx, sy, cy, sz, cz;
    sincos_deg_series(th[3], &sx, &cx);
    sincos_deg_series(th[4], &sy, &cy);
    sincos_deg_series(th[5], &sz, &cz);
    L[0] = dmul(cz, cy);
    L[1] = dadd(-dmul(sz, cx), dmul(dmul(cz, sy), sx));
    L[2] = dadd(dmul(sz, sx), dmul(dmul(cz, sy), cx));
    L[3] = dmul(sz, cy);
    L[4] = dadd(dmul(cz, cx), dmul(dmul(sz, sy), sx));
    L[5] = dadd(-dmul(cz, sx), dmul(dmul(sz, sy), cx));
    L[6] = -sy;
    L[7] = dmul(cy, sx);
    L[8] = dmul(cy, cx);
}

// Affine linear part I + D (D row-major in th[3..11]), each entry one
// rounded addition (an exact copy off the diagonal).
__device__ void affine_linear(const double *th, double L[9])
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) L[3 * r + c] = dadd(r == c ? 1.0 : 0.0, th[3 + 3 * r + c]);
}

__device__ __forceinline__ double dot3_rows(const double *a, double x, double y, double z)
{
    return dadd(dadd(dmul(a[0], x), dmul(a[1], y)), dmul(a[2], z));
}

__device__ __forceinline__ bool quantise(double v, long long *out)
{
    if (!isfinite(v)) return false;
    double s = rint(dmul(v, 1048576.0));
    if (!(fabs(s) < 2147483648.0)) return false;
    *out = (long long)s;
    return true;
}

__global__ void k_pose_to_fixed(const DevGeom *__restrict__ g, const int32_t *__restrict__ desc,
                                const double *__restrict__ poses, int n_params, int n, long long n_pix,
                                int max_side, int kxy, int kz, int32_t *__restrict__ fix,
                                int32_t *__restrict__ err)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t *d = desc + 8 * (size_t)p;
    int32_t *f = fix + kFixStride * (size_t)p;
    int st = d[0], sl = d[1], x0 = d[2], y0 = d[3], w = d[4], h = d[5], off = d[6];
    bool ok = st >= 0 && st < g->n_stacks;
    if (ok) {
        ok = sl >= 0 && sl < g->sk[st] && x0 >= 0 && y0 >= 0 && w >= 1 && h >= 1 &&
             w <= max_side && h <= max_side && x0 + w <= g->sw[st] && y0 + h <= g->sh[st] &&
             off >= 0 && (long long)off + (long long)w * h <= n_pix;
    }
    if (!ok) {
        atomicOr(err, 1);
#pragma unroll
        for (int i = 0; i < kFixStride; ++i) f[i] = 0;
        return;
    }
    const double *th = poses + (size_t)n_params * p;
    const double *S = g->p2w[st];
    const double *W = g->w2v;
    double L[9], c[3], tau[3], A[12], M[12];
    if (n_params == 12)
        affine_linear(th, L);
    else
        rotation_zyx(th, L);
    // patch centre in world
    double u = dadd((double)x0, dmul((double)(w - 1), 0.5));
    double v = dadd((double)y0, dmul((double)(h - 1), 0.5));
    double ks = (double)sl;
    for (int r = 0; r < 3; ++r)
        c[r] = dadd(dot3_rows(S + 4 * r, u, v, ks), S[4 * r + 3]);
    for (int r = 0; r < 3; ++r)
        tau[r] = dsub(dadd(c[r], th[r]), dot3_rows(L + 3 * r, c[0], c[1], c[2]));
    // A = T . S
    for (int r = 0; r < 3; ++r) {
        for (int col = 0; col < 4; ++col)
            A[4 * r + col] = dadd(dadd(dmul(L[3 * r + 0], S[0 * 4 + col]), dmul(L[3 * r + 1], S[1 * 4 + col])),
                                  dmul(L[3 * r + 2], S[2 * 4 + col]));
        A[4 * r + 3] = dadd(A[4 * r + 3], tau[r]);
    }
    // M = W . A
    for (int r = 0; r < 3; ++r) {
        for (int col = 0; col < 4; ++col)
            M[4 * r + col] = dadd(dadd(dmul(W[4 * r + 0], A[0 * 4 + col]), dmul(W[4 * r + 1], A[1 * 4 + col])),
                                  dmul(W[4 * r + 2], A[2 * 4 + col]));
        M[4 * r + 3] = dadd(M[4 * r + 3], W[4 * r + 3]);
    }
    double n2 = dadd(dadd(dmul(S[2], S[2]), dmul(S[6], S[6])), dmul(S[10], S[10]));
    double zs = ddiv(g->dz, __dsqrt_rn(n2));
    double fv[12];
    for (int r = 0; r < 3; ++r) {
        fv[r] = dadd(dadd(dadd(dmul(M[4 * r + 0], (double)x0), dmul(M[4 * r + 1], (double)y0)),
                          dmul(M[4 * r + 2], ks)),
                     M[4 * r + 3]);
        fv[3 + r] = M[4 * r + 0];
        fv[6 + r] = M[4 * r + 1];
        fv[9 + r] = dmul(M[4 * r + 2], zs);
    }
    long long q[12];
    bool good = true;
    bool finite = true;
    for (int i = 0; i < 12; ++i) {
        finite &= (bool)isfinite(fv[i]);
        good &= quantise(fv[i], &q[i]);
    }
    if (!finite) atomicOr(err, 2);
    if (good) {
        long long ci[2] = {-kxy, (long long)(w - 1 + kxy)};
        long long cj[2] = {-kxy, (long long)(h - 1 + kxy)};
        long long cz[2] = {-kz, (long long)kz};
        const long long lim = 1LL << 30;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int z = 0; z < 2; ++z)
                    for (int r = 0; r < 3; ++r) {
                        long long qq = q[r] + ci[a] * q[3 + r] + cj[b] * q[6 + r] + cz[z] * q[9 + r];
                        if (qq > lim || qq < -lim) good = false;
                    }
    }
    for (int i = 0; i < 12; ++i) f[i] = good ? (int32_t)q[i] : 0;
    f[12] = good ? 1 : 0;
    f[13] = 1;   // the descriptor row passed the checks above
    f[14] = f[15] = 0;
}

}  // namespace

cudaError_t launch_pose_to_fixed(const DevGeom *g, const int32_t *desc, const double *poses, int n_params,
                                 int n, int64_t n_pix, int max_side, int kxy, int kz, int32_t *fix,
                                 int32_t *err, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    int bs = 128;
    k_pose_to_fixed<<<(n + bs - 1) / bs, bs, 0, st>>>(g, desc, poses, n_params, n, (long long)n_pix,
                                                      max_side, kxy, kz, fix, err);
    return cudaGetLastError();
}

}  // namespace pvr
