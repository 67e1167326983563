// Host runtime of the warm-start network (include/warmstart.h): parameters, workspace and
// the launch sequences of forward, backward and Adam.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <string>
#include <vector>

#include "subadmm.h"
#include "warmstart.h"
#include "mlp.cuh"
#include "mlp_tc.cuh"
#include "tmap.h"
#include "device_guard.h"

struct wsn_s {
    int device = 0;
    std::vector<int> sizes;            // widths, input .. output
    std::vector<long long> w_off, b_off;
    long long nparams = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // FP32: params, grads, Adam
    __nv_bfloat16 *pb = nullptr;       // BF16 copy of the params
    float *mean = nullptr, *inv_std = nullptr, *scale = nullptr;
    int step = 0;
    // workspace for `cap` rows; its generation is unique in the process and changes with
    // every reallocation (captured graphs that use the workspace check it)
    int cap = 0;
    long long ws_gen = 0;
    std::vector<__nv_bfloat16 *> act;  // act[l]: input of layer l (B x sizes[l])
    std::vector<float *> pre;          // pre[l]: pre-activation of hidden layer l (B x sizes[l+1])
    float *y = nullptr;                // network output (B x out)
    __nv_bfloat16 *g0 = nullptr, *g1 = nullptr;   // layer gradients (B x max width)
    // fused tensor-core inference (the 32-256-256-256-7 warm-start shape): packed BF16
    // weights (K-major per layer), their tensor maps, the kernel's error word
    __nv_bfloat16 *wpack[4] = {nullptr, nullptr, nullptr, nullptr};
    CUtensorMap wmap[4];
    int *ferr = nullptr;
    bool fused_ready = false;
    std::string err;
};

namespace {

std::atomic<long long> g_ws_generation{0};

int werr(wsn_t w, int code, const std::string &msg)
{
    if (w) w->err = msg;
    return code;
}

#define WCK(call, what)                                                             \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) return werr(w, SIM_ECUDA, std::string(what) + ": " + \
                                              cudaGetErrorString(e_));              \
    } while (0)

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4096)); }

void free_ws(wsn_t w)
{
    for (auto *a : w->act) cudaFree(a);
    for (auto *q : w->pre) cudaFree(q);
    w->act.clear();
    w->pre.clear();
    cudaFree(w->y); cudaFree(w->g0); cudaFree(w->g1);
    w->y = nullptr; w->g0 = nullptr; w->g1 = nullptr;
    w->cap = 0;
}

int reserve(wsn_t w, int batch)
{
    if (batch <= w->cap) return SIM_OK;
    free_ws(w);
    const int L = (int)w->sizes.size() - 1;
    const int cap = std::max(batch, 1024);
    int wmax = 0;
    for (int s : w->sizes) wmax = std::max(wmax, s);
    w->act.assign(L, nullptr);
    w->pre.assign(L, nullptr);
    for (int l = 0; l < L; ++l) {
        WCK(cudaMalloc((void **)&w->act[l], sizeof(__nv_bfloat16) * (size_t)cap * w->sizes[l]), "cudaMalloc");
        WCK(cudaMalloc((void **)&w->pre[l], sizeof(float) * (size_t)cap * w->sizes[l + 1]), "cudaMalloc");
    }
    WCK(cudaMalloc((void **)&w->y, sizeof(float) * (size_t)cap * w->sizes[L]), "cudaMalloc");
    WCK(cudaMalloc((void **)&w->g0, sizeof(__nv_bfloat16) * (size_t)cap * wmax), "cudaMalloc");
    WCK(cudaMalloc((void **)&w->g1, sizeof(__nv_bfloat16) * (size_t)cap * wmax), "cudaMalloc");
    w->cap = cap;
    w->ws_gen = ++g_ws_generation;
    return SIM_OK;
}

template <int EPI>
int gemm(wsn_t w, const wsn::Gemm &g, cudaStream_t st)
{
    dim3 grid((g.N + wsn::TN - 1) / wsn::TN, (g.M + wsn::TM - 1) / wsn::TM);
    wsn::gemm_kernel<EPI><<<grid, 128, 0, st>>>(g);
    WCK(cudaGetLastError(), "gemm launch");
    return SIM_OK;
}

// forward over `batch` rows; the network's raw output in w->y (scaled by scale_out when
// `scaled`); inputs and hidden activations kept for backward
int forward(wsn_t w, const float *x, long long ldx, int batch, bool scaled, cudaStream_t st)
{
    int rc = reserve(w, batch);
    if (rc) return rc;
    const int L = (int)w->sizes.size() - 1;
    wsn::normalize_kernel<<<grid_for((long long)batch * w->sizes[0]), 256, 0, st>>>(
        x, ldx, w->mean, w->inv_std, w->act[0], batch, w->sizes[0]);
    WCK(cudaGetLastError(), "normalize launch");
    for (int l = 0; l < L; ++l) {
        wsn::Gemm g{};
        g.A = w->act[l]; g.sam = w->sizes[l]; g.sak = 1;
        g.B = w->pb + w->w_off[l]; g.sbk = w->sizes[l + 1]; g.sbn = 1;
        g.M = batch; g.N = w->sizes[l + 1]; g.K = w->sizes[l];
        g.bias = w->p + w->b_off[l];
        if (l < L - 1) {
            g.out = w->pre[l];
            g.act = w->act[l + 1];
            if ((rc = gemm<wsn::EPI_BIAS_GELU>(w, g, st))) return rc;
        } else {
            g.out = w->y;
            g.scale = scaled ? w->scale : nullptr;
            if ((rc = gemm<wsn::EPI_BIAS>(w, g, st))) return rc;
        }
    }
    return SIM_OK;
}

// backward from w->y against t (output units): gradients into grad (parameter order)
int backward(wsn_t w, const float *t, const float *mask, int batch, float *grad, float *loss,
             cudaStream_t st)
{
    const int L = (int)w->sizes.size() - 1;
    const int N = w->sizes[L];
    wsn::output_grad_kernel<<<grid_for((long long)batch * N), 256, 0, st>>>(
        w->y, t, mask, w->scale, w->g0, batch, N, loss);
    WCK(cudaGetLastError(), "output grad launch");
    __nv_bfloat16 *gcur = w->g0, *gnext = w->g1;
    int rc;
    for (int l = L - 1; l >= 0; --l) {
        const int in = w->sizes[l], out = w->sizes[l + 1];
        wsn::Gemm gw{};                         // dW = act^T g
        gw.A = w->act[l]; gw.sam = 1; gw.sak = in;
        gw.B = gcur; gw.sbk = out; gw.sbn = 1;
        gw.M = in; gw.N = out; gw.K = batch;
        gw.out = grad + w->w_off[l];
        if ((rc = gemm<wsn::EPI_STORE>(w, gw, st))) return rc;
        wsn::column_sum_kernel<<<(out + 31) / 32, 256, 0, st>>>(gcur, batch, out, grad + w->b_off[l]);
        WCK(cudaGetLastError(), "column sum launch");
        if (l > 0) {                            // g_prev = (g W^T) * GELU'(pre)
            wsn::Gemm ga{};
            ga.A = gcur; ga.sam = out; ga.sak = 1;
            ga.B = w->pb + w->w_off[l]; ga.sbk = 1; ga.sbn = out;
            ga.M = batch; ga.N = in; ga.K = out;
            ga.pre = w->pre[l - 1];
            ga.act = gnext;
            if ((rc = gemm<wsn::EPI_GELU_BWD>(w, ga, st))) return rc;
            std::swap(gcur, gnext);
        }
    }
    return SIM_OK;
}

}  // namespace

namespace {

bool fused_shape(const wsn_t w)
{
    return w->sizes.size() == 5 && w->sizes[0] == wsn::kMlpIn && w->sizes[1] == wsn::kMlpHidden &&
           w->sizes[2] == wsn::kMlpHidden && w->sizes[3] == wsn::kMlpHidden &&
           w->sizes[4] == wsn::kMlpOut;
}

// the warm-start shape: pack the current BF16 weights (every call, so that a captured graph
// sees parameters trained after its capture) and run all four layers in one launch
int fused_forward(wsn_t w, const float *x, long long ldx, int batch, float *y, cudaStream_t st)
{
    using namespace wsn;
    if (!w->fused_ready) {
        const size_t n[4] = {(size_t)kMlpHidden * kMlpInPad, (size_t)kMlpHidden * kMlpHidden,
                             (size_t)kMlpHidden * kMlpHidden, (size_t)kMlpOutPad * kMlpHidden};
        const int inner[4] = {kMlpInPad, kMlpHidden, kMlpHidden, kMlpHidden};
        const int rows[4] = {kMlpHidden, kMlpHidden, kMlpHidden, kMlpOutPad};
        for (int l = 0; l < 4; ++l) {
            WCK(cudaMalloc((void **)&w->wpack[l], sizeof(__nv_bfloat16) * n[l]), "cudaMalloc packed weights");
            WCK(subadmm::tmap_encode_2d(&w->wmap[l], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                                        sizeof(__nv_bfloat16), w->wpack[l], inner[l], rows[l], 64,
                                        rows[l]), "tensor map");
        }
        WCK(cudaMalloc((void **)&w->ferr, sizeof(int)), "cudaMalloc error word");
        WCK(cudaMemset(w->ferr, 0, sizeof(int)), "error word");
        WCK(cudaFuncSetAttribute((const void *)mlp_fused_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kMlpSmem), "attribute");
        w->fused_ready = true;
    }
    mlp_pack_kernel<<<256, 256, 0, st>>>(w->pb, w->w_off[0], w->w_off[1], w->w_off[2], w->w_off[3],
                                         w->wpack[0], w->wpack[1], w->wpack[2], w->wpack[3]);
    WCK(cudaGetLastError(), "pack launch");
    MlpArgs a;
    a.x = x; a.ldx = ldx; a.batch = batch; a.mean = w->mean; a.inv_std = w->inv_std;
    for (int l = 0; l < 4; ++l) a.bias[l] = w->p + w->b_off[l];
    a.scale = w->scale; a.y = y; a.err = w->ferr;
    int sms = 0;
    WCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, w->device), "attribute");
    const int tiles = (batch + kMlpRows - 1) / kMlpRows;
    mlp_fused_kernel<<<std::max(1, std::min(tiles, sms)), kMlpThreads, kMlpSmem, st>>>(
        w->wmap[0], w->wmap[1], w->wmap[2], w->wmap[3], a);
    WCK(cudaGetLastError(), "fused forward launch");
    return SIM_OK;
}

}  // namespace

extern "C" {

int wsn_create(int device, int n_layers, const int *sizes, wsn_t *out)
{
    if (!out || !sizes || n_layers < 1) return SIM_EINVAL;
    *out = nullptr;
    for (int l = 0; l <= n_layers; ++l)
        if (sizes[l] < 1 || sizes[l] > 1024) return SIM_EINVAL;
    subadmm::DeviceGuard on_device(device);
    if (on_device.err != cudaSuccess) return SIM_ECUDA;
    wsn_t w = new wsn_s();
    w->device = device;
    w->sizes.assign(sizes, sizes + n_layers + 1);
    long long off = 0;
    for (int l = 0; l < n_layers; ++l) {
        w->w_off.push_back(off);
        off += (long long)sizes[l] * sizes[l + 1];
        w->b_off.push_back(off);
        off += sizes[l + 1];
    }
    w->nparams = off;
    const size_t bytes = sizeof(float) * (size_t)off;
    bool ok = cudaMalloc((void **)&w->p, bytes) == cudaSuccess &&
              cudaMalloc((void **)&w->g, bytes) == cudaSuccess &&
              cudaMalloc((void **)&w->m, bytes) == cudaSuccess &&
              cudaMalloc((void **)&w->v, bytes) == cudaSuccess &&
              cudaMalloc((void **)&w->pb, sizeof(__nv_bfloat16) * (size_t)off) == cudaSuccess &&
              cudaMalloc((void **)&w->mean, sizeof(float) * sizes[0]) == cudaSuccess &&
              cudaMalloc((void **)&w->inv_std, sizeof(float) * sizes[0]) == cudaSuccess &&
              cudaMalloc((void **)&w->scale, sizeof(float) * sizes[n_layers]) == cudaSuccess;
    if (!ok) { wsn_destroy(w); return SIM_ENOMEM; }
    cudaMemset(w->p, 0, bytes);
    cudaMemset(w->m, 0, bytes);
    cudaMemset(w->v, 0, bytes);
    cudaMemset(w->pb, 0, sizeof(__nv_bfloat16) * (size_t)off);
    std::vector<float> zeros(sizes[0], 0.0f), ones(std::max(sizes[0], sizes[n_layers]), 1.0f);
    cudaMemcpy(w->mean, zeros.data(), sizeof(float) * sizes[0], cudaMemcpyHostToDevice);
    cudaMemcpy(w->inv_std, ones.data(), sizeof(float) * sizes[0], cudaMemcpyHostToDevice);
    cudaMemcpy(w->scale, ones.data(), sizeof(float) * sizes[n_layers], cudaMemcpyHostToDevice);
    if (cudaDeviceSynchronize() != cudaSuccess) { wsn_destroy(w); return SIM_ECUDA; }
    *out = w;
    return SIM_OK;
}

void wsn_destroy(wsn_t w)
{
    if (!w) return;
    subadmm::DeviceGuard on_device(w->device);
    free_ws(w);
    for (auto *q : w->wpack) cudaFree(q);
    cudaFree(w->ferr);
    cudaFree(w->p); cudaFree(w->g); cudaFree(w->m); cudaFree(w->v); cudaFree(w->pb);
    cudaFree(w->mean); cudaFree(w->inv_std); cudaFree(w->scale);
    delete w;
}

const char *wsn_last_error(wsn_t w) { return w ? w->err.c_str() : ""; }

long long wsn_num_params(wsn_t w) { return w ? w->nparams : -1; }

long long wsn_workspace_generation(wsn_t w) { return w ? w->ws_gen : -1; }

int wsn_shape(wsn_t w, int shape[2])
{
    if (!w || !shape) return SIM_EINVAL;
    shape[0] = w->sizes.front();
    shape[1] = w->sizes.back();
    return SIM_OK;
}

int wsn_set_params(wsn_t w, const float *params)
{
    if (!w || !params) return SIM_EINVAL;
    subadmm::DeviceGuard on_device(w->device);
    WCK(on_device.err, "cudaSetDevice");
    const size_t bytes = sizeof(float) * (size_t)w->nparams;
    WCK(cudaMemcpy(w->p, params, bytes, cudaMemcpyHostToDevice), "params");
    WCK(cudaMemset(w->m, 0, bytes), "adam state");
    WCK(cudaMemset(w->v, 0, bytes), "adam state");
    w->step = 0;
    wsn::to_bf16_kernel<<<grid_for(w->nparams), 256>>>(w->p, w->pb, w->nparams);
    WCK(cudaGetLastError(), "bf16 copy");
    WCK(cudaDeviceSynchronize(), "synchronize");
    return SIM_OK;
}

int wsn_get_params(wsn_t w, float *params)
{
    if (!w || !params) return SIM_EINVAL;
    subadmm::DeviceGuard on_device(w->device);
    WCK(on_device.err, "cudaSetDevice");
    WCK(cudaDeviceSynchronize(), "synchronize");
    WCK(cudaMemcpy(params, w->p, sizeof(float) * (size_t)w->nparams, cudaMemcpyDeviceToHost), "params");
    return SIM_OK;
}

int wsn_set_normalization(wsn_t w, const float *mean_in, const float *std_in,
                          const float *scale_out)
{
    if (!w || !mean_in || !std_in || !scale_out) return SIM_EINVAL;
    const int D = w->sizes[0], N = w->sizes.back();
    std::vector<float> inv(D);
    for (int d = 0; d < D; ++d) {
        if (!(std_in[d] > 0.0f)) return werr(w, SIM_EINVAL, "std_in must be > 0");
        inv[d] = 1.0f / std_in[d];
    }
    subadmm::DeviceGuard on_device(w->device);
    WCK(on_device.err, "cudaSetDevice");
    WCK(cudaMemcpy(w->mean, mean_in, sizeof(float) * D, cudaMemcpyHostToDevice), "mean");
    WCK(cudaMemcpy(w->inv_std, inv.data(), sizeof(float) * D, cudaMemcpyHostToDevice), "std");
    WCK(cudaMemcpy(w->scale, scale_out, sizeof(float) * N, cudaMemcpyHostToDevice), "scale");
    return SIM_OK;
}

int wsn_get_normalization(wsn_t w, float *mean_in, float *std_in, float *scale_out)
{
    if (!w || !mean_in || !std_in || !scale_out) return SIM_EINVAL;
    const int D = w->sizes[0], N = w->sizes.back();
    std::vector<float> inv(D);
    subadmm::DeviceGuard on_device(w->device);
    WCK(on_device.err, "cudaSetDevice");
    WCK(cudaDeviceSynchronize(), "synchronize");
    WCK(cudaMemcpy(mean_in, w->mean, sizeof(float) * D, cudaMemcpyDeviceToHost), "mean");
    WCK(cudaMemcpy(inv.data(), w->inv_std, sizeof(float) * D, cudaMemcpyDeviceToHost), "std");
    WCK(cudaMemcpy(scale_out, w->scale, sizeof(float) * N, cudaMemcpyDeviceToHost), "scale");
    for (int d = 0; d < D; ++d) std_in[d] = 1.0f / inv[d];
    return SIM_OK;
}

int wsn_fit_normalization(wsn_t w, const float *x_dev, long long ldx, const float *t_dev,
                          int batch, void *stream)
{
    if (!w || !x_dev || !t_dev || batch < 1 || ldx < w->sizes[0]) return SIM_EINVAL;
    subadmm::DeviceGuard on_device(w->device);
    WCK(on_device.err, "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int D = w->sizes[0], N = w->sizes.back();
    wsn::column_stats_kernel<<<D, 256, 0, st>>>(x_dev, ldx, batch, D, w->mean, w->inv_std, 1);
    WCK(cudaGetLastError(), "stats launch");
    wsn::column_stats_kernel<<<N, 256, 0, st>>>(t_dev, N, batch, N, nullptr, w->scale, 0);
    WCK(cudaGetLastError(), "stats launch");
    return SIM_OK;
}

int wsn_fused_error(wsn_t w, int *out)
{
    if (!w || !out) return SIM_EINVAL;
    *out = 0;
    if (!w->ferr) return SIM_OK;
    subadmm::DeviceGuard on_device(w->device);
    WCK(on_device.err, "cudaSetDevice");
    WCK(cudaMemcpy(out, w->ferr, sizeof(int), cudaMemcpyDeviceToHost), "error word");
    WCK(cudaMemset(w->ferr, 0, sizeof(int)), "error word");
    return SIM_OK;
}

int wsn_forward_layers(wsn_t w, const float *x_dev, long long ldx, int batch,
                                  float *y_dev, void *stream)
{
    if (!w || !x_dev || !y_dev || batch < 0 || ldx < w->sizes[0]) return SIM_EINVAL;
    if (batch == 0) return SIM_OK;
    subadmm::DeviceGuard on_device(w->device);
    WCK(on_device.err, "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = forward(w, x_dev, ldx, batch, true, st);
    if (rc) return rc;
    WCK(cudaMemcpyAsync(y_dev, w->y, sizeof(float) * (size_t)batch * w->sizes.back(),
                        cudaMemcpyDeviceToDevice, st), "output copy");
    return SIM_OK;
}

int wsn_forward(wsn_t w, const float *x_dev, long long ldx, int batch, float *y_dev, void *stream)
{
    if (!w || !x_dev || !y_dev || batch < 0 || ldx < w->sizes[0]) return SIM_EINVAL;
    if (batch == 0) return SIM_OK;
    subadmm::DeviceGuard on_device(w->device);
    WCK(on_device.err, "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (fused_shape(w)) return fused_forward(w, x_dev, ldx, batch, y_dev, st);
    int rc = forward(w, x_dev, ldx, batch, true, st);
    if (rc) return rc;
    WCK(cudaMemcpyAsync(y_dev, w->y, sizeof(float) * (size_t)batch * w->sizes.back(),
                        cudaMemcpyDeviceToDevice, st), "output copy");
    return SIM_OK;
}

int wsn_gradients(wsn_t w, const float *x_dev, long long ldx, const float *t_dev,
                  const float *mask_dev, int batch, float *grad_dev, float *loss_dev,
                  void *stream)
{
    if (!w || !x_dev || !t_dev || !mask_dev || !grad_dev || batch < 1 || ldx < w->sizes[0])
        return SIM_EINVAL;
    subadmm::DeviceGuard on_device(w->device);
    WCK(on_device.err, "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = forward(w, x_dev, ldx, batch, false, st);
    if (rc) return rc;
    return backward(w, t_dev, mask_dev, batch, grad_dev, loss_dev, st);
}

int wsn_train_step(wsn_t w, const float *x_dev, long long ldx, const float *t_dev,
                   const float *mask_dev, int batch, float lr, float *loss_dev, void *stream)
{
    int rc = wsn_gradients(w, x_dev, ldx, t_dev, mask_dev, batch, w ? w->g : nullptr, loss_dev, stream);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    w->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)w->step), c2 = 1.0f - std::pow(b2, (float)w->step);
    wsn::adam_kernel<<<grid_for(w->nparams), 256, 0, st>>>(w->p, w->pb, w->g, w->m, w->v, w->nparams,
                                                            lr, b1, b2, 1e-8f, c1, c2);
    WCK(cudaGetLastError(), "adam launch");
    return SIM_OK;
}

}  // extern "C"
