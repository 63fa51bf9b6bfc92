// pvr_net: the learned pose proposal.  A 2-D CNN reads a 64x64 acquired
// patch and the patch simulated at the current pose estimate and predicts
// the rigid correction (6 parameters, in the frame of the patch's stack:
// along / about its column, row and normal directions) that registers them; NCC registration
// starts from the proposal where it improves NCC and from the plain pose
// otherwise.  Six 3x3 convolutions (ReLU; 32, 32, 64, 64, 64, 64 channels;
// strides 1, 2, 2, 2, 2, 1) and a linear head on the flattened 4x4x64
// last activation (positions kept: a mean over them would discard where
// the patch content lies, and with it the in-plane translation).
// Weights: float32 master copies with Adam moments, bfloat16 working copies
// for the tensor-core convolutions (csrc/k_cnn.cu).
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <random>
#include <vector>

#include "pvr_internal.h"

namespace pvr {
cudaError_t cnn_conv_forward(const __nv_bfloat16 *in, const __nv_bfloat16 *w, const float *bias,
                             __nv_bfloat16 *out, int B, int IH, int IW, int Cin, int Cout, int stride,
                             cudaStream_t st);
cudaError_t cnn_conv_backward(const __nv_bfloat16 *in, const __nv_bfloat16 *w, const __nv_bfloat16 *out,
                              const __nv_bfloat16 *gout, __nv_bfloat16 *gin, float *gw, float *gb, int B,
                              int IH, int IW, int Cin, int Cout, int stride, cudaStream_t st);
cudaError_t cnn_input(const float *y, const float *s, const uint8_t *valid, const int32_t *desc, int first,
                      int count, int64_t n_pix, __nv_bfloat16 *img, cudaStream_t st);
cudaError_t cnn_head_forward(const __nv_bfloat16 *act, int B, int F, const float *wl, const float *bl, int J,
                             float *feat, float *out, cudaStream_t st);
cudaError_t cnn_head_backward(const float *out, const float *target, int B, int J, const float *feat,
                              const float *wl, int F, float *gwl, float *gbl, __nv_bfloat16 *gact,
                              float *loss, cudaStream_t st);
cudaError_t cnn_adam(float *w, const float *gw, float *m1, float *m2, long long n, float lr, int step,
                     __nv_bfloat16 *wb, cudaStream_t st);
cudaError_t cnn_to_bf16(const float *a, __nv_bfloat16 *b, long long n, cudaStream_t st);
cudaError_t cnn_propose_trial(const DevGeom *g, const int32_t *desc, const double *poses, const float *out, int n,
                              const double scale[6], double *trial, cudaStream_t st);
cudaError_t cnn_read_timeout(unsigned *host_flag, cudaStream_t st);
cudaError_t cnn_propose_select(const double *ncc0, const double *ncc1, const double *trial, int n, double *poses,
                               int32_t *accepted, cudaStream_t st);
}  // namespace pvr

using namespace pvr;

namespace {

struct Layer {
    int Cin, Cout, stride, IH;   // square images
    int OH() const { return (IH - 1) / stride + 1; }
    long long nw() const { return (long long)Cout * 9 * Cin; }
};

const Layer kLayers[] = {{16, 32, 1, 64}, {32, 32, 2, 64}, {32, 64, 2, 32},
                         {64, 64, 2, 16}, {64, 64, 2, 8},  {64, 64, 1, 4}};
constexpr int kNL = 6, kSide = 64, kInC = 16, kOut = 6;
constexpr int kFeat = 4 * 4 * 64;   // flattened last activation (OH x OW x Cout of the last layer)

}  // namespace

struct pvr_net {
    int batch_max = 0;
    long long n_params = 0;
    long long w_off[kNL], b_off[kNL], head_w = 0, head_b = 0;
    float *w = nullptr, *gw = nullptr, *m1 = nullptr, *m2 = nullptr;
    __nv_bfloat16 *wb = nullptr;
    __nv_bfloat16 *img = nullptr, *act[kNL] = {}, *gact[kNL] = {};
    float *pooled = nullptr, *out = nullptr, *loss = nullptr;   // pooled: head features [batch][kFeat]
    int step = 0;
    // scratch of pvr_pose_propose (pvr_net_reserve)
    int64_t res_patches = 0, res_pixels = 0;
    float *sim = nullptr, *props = nullptr;
    uint8_t *valid = nullptr;
    double *trial = nullptr, *ncc = nullptr;
};

namespace {

void net_free(pvr_net *n)
{
    void *p[] = {n->w, n->gw, n->m1, n->m2, n->wb, n->img, n->pooled, n->out, n->loss,
                 n->sim, n->props, n->valid, n->trial, n->ncc};
    for (void *q : p)
        if (q) cudaFree(q);
    for (int l = 0; l < kNL; ++l) {
        if (n->act[l]) cudaFree(n->act[l]);
        if (n->gact[l]) cudaFree(n->gact[l]);
    }
}

bool table_ok(const pvr_patches *pp, int first, int count, int batch_max)
{
    return pp && pp->desc && count >= 1 && count <= batch_max && first >= 0 && first + count <= pp->n &&
           pp->max_side == kSide;
}

int forward(pvr_net *n, const float *y, const float *s, const uint8_t *valid, const pvr_patches *pp, int first,
            int count, cudaStream_t st)
{
    if (cnn_input(y, s, valid, pp->desc, first, count, pp->n_pix, n->img, st) != cudaSuccess) return PVR_ERR_CUDA;
    const __nv_bfloat16 *in = n->img;
    for (int l = 0; l < kNL; ++l) {
        const Layer &L = kLayers[l];
        if (cnn_conv_forward(in, n->wb + n->w_off[l], n->w + n->b_off[l], n->act[l], count, L.IH, L.IH, L.Cin,
                             L.Cout, L.stride, st) != cudaSuccess)
            return PVR_ERR_CUDA;
        in = n->act[l];
    }
    if (cnn_head_forward(n->act[kNL - 1], count, kFeat, n->w + n->head_w, n->w + n->head_b, kOut, n->pooled,
                         n->out, st) != cudaSuccess)
        return PVR_ERR_CUDA;
    return PVR_OK;
}

}  // namespace

extern "C" {

PVR_API int pvr_net_create(pvr_net **out, int32_t batch_max, uint64_t seed)
{
    if (!out || batch_max < 1 || batch_max > 4096) return PVR_ERR_INVALID_ARG;
    *out = nullptr;
    pvr_net *n = new pvr_net();
    n->batch_max = batch_max;
    long long o = 0;
    for (int l = 0; l < kNL; ++l) {
        n->w_off[l] = o;
        o += kLayers[l].nw();
        n->b_off[l] = o;
        o += kLayers[l].Cout;
    }
    n->head_w = o;
    o += (long long)kOut * kFeat;
    n->head_b = o;
    o += kOut;
    n->n_params = o;
    // He-normal convolutions (fan-in over the two real input channels of
    // the first layer), small head, zero biases
    std::vector<float> h((size_t)o, 0.f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < kNL; ++l) {
        const Layer &L = kLayers[l];
        const int cin_real = l == 0 ? 2 : L.Cin;
        std::normal_distribution<float> nd(0.f, sqrtf(2.f / (9.f * cin_real)));
        for (int co = 0; co < L.Cout; ++co)
            for (int t = 0; t < 9; ++t)
                for (int ci = 0; ci < L.Cin; ++ci)
                    h[(size_t)(n->w_off[l] + ((long long)co * 9 + t) * L.Cin + ci)] = ci < cin_real ? nd(rng) : 0.f;
    }
    std::normal_distribution<float> nh(0.f, 0.01f);
    for (long long i = n->head_w; i < n->head_b; ++i) h[(size_t)i] = nh(rng);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes > 0 ? bytes : 1);
    };
    alloc((void **)&n->w, o * sizeof(float));
    alloc((void **)&n->gw, o * sizeof(float));
    alloc((void **)&n->m1, o * sizeof(float));
    alloc((void **)&n->m2, o * sizeof(float));
    alloc((void **)&n->wb, o * sizeof(__nv_bfloat16));
    alloc((void **)&n->img, (size_t)batch_max * kSide * kSide * kInC * sizeof(__nv_bfloat16));
    for (int l = 0; l < kNL; ++l) {
        const Layer &L = kLayers[l];
        const size_t sz = (size_t)batch_max * L.OH() * L.OH() * L.Cout * sizeof(__nv_bfloat16);
        alloc((void **)&n->act[l], sz);
        alloc((void **)&n->gact[l], sz);
    }
    alloc((void **)&n->pooled, (size_t)batch_max * kFeat * sizeof(float));
    alloc((void **)&n->out, (size_t)batch_max * kOut * sizeof(float));
    alloc((void **)&n->loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(n->w, h.data(), o * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(n->m1, 0, o * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(n->m2, 0, o * sizeof(float));
    if (e == cudaSuccess) e = cnn_to_bf16(n->w, n->wb, o, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        net_free(n);
        delete n;
        return PVR_ERR_CUDA;
    }
    *out = n;
    return PVR_OK;
}

PVR_API int pvr_net_destroy(pvr_net *n)
{
    if (!n) return PVR_OK;
    cudaDeviceSynchronize();
    net_free(n);
    delete n;
    return PVR_OK;
}

PVR_API int64_t pvr_net_param_count(const pvr_net *n) { return n ? n->n_params : 0; }

PVR_API int pvr_net_get_params(pvr_net *n, float *host)
{
    if (!n || !host) return PVR_ERR_INVALID_ARG;
    return cudaMemcpy(host, n->w, n->n_params * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess
               ? PVR_OK
               : PVR_ERR_CUDA;
}

PVR_API int pvr_net_set_params(pvr_net *n, const float *host)
{
    if (!n || !host) return PVR_ERR_INVALID_ARG;
    if (cudaMemcpy(n->w, host, n->n_params * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return PVR_ERR_CUDA;
    if (cnn_to_bf16(n->w, n->wb, n->n_params, 0) != cudaSuccess) return PVR_ERR_CUDA;
    n->step = 0;
    cudaMemset(n->m1, 0, n->n_params * sizeof(float));
    cudaMemset(n->m2, 0, n->n_params * sizeof(float));
    return cudaDeviceSynchronize() == cudaSuccess ? PVR_OK : PVR_ERR_CUDA;
}

PVR_API int pvr_net_forward(pvr_net *n, const float *y, const float *s, const uint8_t *valid, const pvr_patches *pp,
                    int32_t first, int32_t count, float *out, void *stream)
{
    if (!n || !y || !s || !valid || !out || !table_ok(pp, first, count, n->batch_max)) return PVR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = forward(n, y, s, valid, pp, first, count, st);
    if (rc) return rc;
    return cudaMemcpyAsync(out, n->out, (size_t)count * kOut * sizeof(float), cudaMemcpyDeviceToDevice, st) ==
                   cudaSuccess
               ? PVR_OK
               : PVR_ERR_CUDA;
}

PVR_API int pvr_net_train_step(pvr_net *n, const float *y, const float *s, const uint8_t *valid, const pvr_patches *pp,
                       int32_t first, int32_t count, const float *target, float lr, float *loss, void *stream)
{
    if (!n || !y || !s || !valid || !target || !table_ok(pp, first, count, n->batch_max) || !(lr > 0.f))
        return PVR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(n->gw, 0, n->n_params * sizeof(float), st) != cudaSuccess) return PVR_ERR_CUDA;
    if (cudaMemsetAsync(n->loss, 0, sizeof(float), st) != cudaSuccess) return PVR_ERR_CUDA;
    int rc = forward(n, y, s, valid, pp, first, count, st);
    if (rc) return rc;
    if (cnn_head_backward(n->out, target, count, kOut, n->pooled, n->w + n->head_w, kFeat, n->gw + n->head_w,
                          n->gw + n->head_b, n->gact[kNL - 1], n->loss, st) != cudaSuccess)
        return PVR_ERR_CUDA;
    for (int l = kNL - 1; l >= 0; --l) {
        const Layer &L = kLayers[l];
        const __nv_bfloat16 *in = l == 0 ? n->img : n->act[l - 1];
        __nv_bfloat16 *gin = l == 0 ? nullptr : n->gact[l - 1];
        if (cnn_conv_backward(in, n->wb + n->w_off[l], n->act[l], n->gact[l], gin, n->gw + n->w_off[l],
                              n->gw + n->b_off[l], count, L.IH, L.IH, L.Cin, L.Cout, L.stride, st) != cudaSuccess)
            return PVR_ERR_CUDA;
    }
    ++n->step;
    if (cnn_adam(n->w, n->gw, n->m1, n->m2, n->n_params, lr, n->step, n->wb, st) != cudaSuccess) return PVR_ERR_CUDA;
    if (loss && cudaMemcpyAsync(loss, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return PVR_ERR_CUDA;
    return PVR_OK;
}

PVR_API int pvr_net_reserve(pvr_net *n, int32_t max_patches, int64_t max_pixels)
{
    if (!n || max_patches < 1 || max_pixels < 1) return PVR_ERR_INVALID_ARG;
    void *p[] = {n->sim, n->props, n->valid, n->trial, n->ncc};
    for (void *q : p)
        if (q) cudaFree(q);
    n->sim = n->props = nullptr;
    n->valid = nullptr;
    n->trial = n->ncc = nullptr;
    n->res_patches = n->res_pixels = 0;
    cudaError_t e = cudaMalloc((void **)&n->sim, (size_t)max_pixels * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&n->valid, (size_t)max_pixels);
    if (e == cudaSuccess) e = cudaMalloc((void **)&n->props, (size_t)max_patches * kOut * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&n->trial, (size_t)max_patches * 6 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&n->ncc, (size_t)max_patches * 2 * sizeof(double));
    if (e != cudaSuccess) return PVR_ERR_CUDA;
    n->res_patches = max_patches;
    n->res_pixels = max_pixels;
    return PVR_OK;
}

PVR_API int pvr_pose_propose(pvr_ctx *ctx, pvr_net *n, const float *x, const float *y, const pvr_patches *pp,
                             const double *scale, double *poses, int32_t *accepted, void *stream)
{
    if (!ctx || !n || !pp || !scale) return PVR_ERR_INVALID_ARG;
    if (ctx_n_params(ctx) != 6) return PVR_ERR_UNSUPPORTED;   // the network predicts rigid corrections
    if (pp->n == 0) return PVR_OK;
    if (!x || !y || !poses || pp->max_side != kSide) return PVR_ERR_INVALID_ARG;
    if (pp->n > n->res_patches || pp->n_pix > n->res_pixels) return PVR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    // the patches simulated at the current poses, the network's corrections
    if ((rc = pvr_simulate(ctx, x, pp, poses, n->sim, n->valid, stream))) return rc;
    for (int first = 0; first < pp->n; first += n->batch_max) {
        const int cnt = pp->n - first < n->batch_max ? pp->n - first : n->batch_max;
        if ((rc = pvr_net_forward(n, y, n->sim, n->valid, pp, first, cnt, n->props + (size_t)first * kOut, stream)))
            return rc;
    }
    if (cnn_propose_trial(ctx_dev_geom(ctx), pp->desc, poses, n->props, pp->n, scale, n->trial, st) != cudaSuccess)
        return PVR_ERR_CUDA;
    // NCC at the plain and at the proposed pose; keep the better
    if ((rc = pvr_ncc_grad(ctx, x, y, pp, poses, n->ncc, nullptr, stream))) return rc;
    if ((rc = pvr_ncc_grad(ctx, x, y, pp, n->trial, n->ncc + pp->n, nullptr, stream))) return rc;
    if (cnn_propose_select(n->ncc, n->ncc + pp->n, n->trial, pp->n, poses, accepted, st) != cudaSuccess)
        return PVR_ERR_CUDA;
    return PVR_OK;
}

PVR_API int pvr_net_status(pvr_net *n, void *stream)
{
    if (!n) return PVR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned h = 0;
    if (cnn_read_timeout(&h, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return PVR_ERR_CUDA;
    return h ? PVR_ERR_TIMEOUT : PVR_OK;
}

// Gradients of the last train step (float32, layout of pvr_net_get_params).
PVR_API int pvr_net_get_grads(pvr_net *n, float *host)
{
    if (!n || !host) return PVR_ERR_INVALID_ARG;
    return cudaMemcpy(host, n->gw, n->n_params * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess
               ? PVR_OK
               : PVR_ERR_CUDA;
}

}  // extern "C"
