// Host side of the surrogate network (morea_mlp_*): parameter storage, the
// forward pass, the gradients and the Adam step, all on the stream given.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "morea_host.h"
#include "morea_mlp.h"

using namespace morea;

struct morea_mlp {
    int device = 0;
    int n_in = 0, h1 = 0, h2 = 0, n_out = 0, max_batch = 0;
    int kin = 0, bpad = 0;                 // padded input width (x64) and batch (x32)
    long long n_params = 0;                // W1 [h1][kin], b1, W2 [h2][h1], b2, W3 [n_out][h2], b3
    long long oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
    std::vector<void *> allocs;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // FP32 params, grads, Adam moments
    void *W1b = nullptr, *W2b = nullptr, *W2Tb = nullptr, *W3b = nullptr;
    void *X = nullptr, *XT = nullptr, *H1 = nullptr, *H1T = nullptr, *H2 = nullptr;
    void *dH2 = nullptr, *dH2T = nullptr, *dH1 = nullptr, *dH1T = nullptr;
    float *Y = nullptr, *dY = nullptr, *loss = nullptr;
    int *status = nullptr;                 // device status word (bit 0: a GEMM wait gave up)
    float *ws = nullptr;                   // split-K workspace of the tensor-core products
    long long ws_floats = 0;
    long long step = 0;
};

namespace {

morea_status from_cuda(cudaError_t e) { return e == cudaSuccess ? MOREA_OK : MOREA_ECUDA; }

inline long long up(long long x, long long a) { return (x + a - 1) / a * a; }

// BF16 working copies of the weights (and the transposed W2 for dH1).
cudaError_t refresh_bf16(morea_mlp *n, cudaStream_t st)
{
    cudaError_t e = mlp_cast((long long)n->h1 * n->kin, n->w + n->oW1, n->W1b, st);
    if (e == cudaSuccess) e = mlp_cast((long long)n->h2 * n->h1, n->w + n->oW2, n->W2b, st);
    if (e == cudaSuccess) e = mlp_cast((long long)n->n_out * n->h2, n->w + n->oW3, n->W3b, st);
    if (e == cudaSuccess) e = mlp_transpose(n->h2, n->h1, n->h2, n->W2b, n->h1, n->W2Tb, n->h2, st);
    return e;
}

cudaError_t forward(morea_mlp *n, int b, const float *x, cudaStream_t st)
{
    cudaError_t e = mlp_to_bf16(b, n->n_in, b, n->kin, x, n->X, st);
    if (e == cudaSuccess)
        e = mlp_gemm_nt(b, n->h1, n->kin, n->X, n->kin, n->W1b, n->kin, n->w + n->ob1, nullptr, 0, 1, nullptr, 0,
                        n->H1, n->h1, n->ws, n->ws_floats, n->status, st);
    if (e == cudaSuccess)
        e = mlp_gemm_nt(b, n->h2, n->h1, n->H1, n->h1, n->W2b, n->h1, n->w + n->ob2, nullptr, 0, 1, nullptr, 0,
                        n->H2, n->h2, n->ws, n->ws_floats, n->status, st);
    if (e == cudaSuccess) e = mlp_out_fwd(b, n->h2, n->n_out, n->H2, n->h2, n->W3b, n->h2, n->w + n->ob3, n->Y, st);
    return e;
}

// Gradient of the mean squared error of batch (x, t) into n->g.
cudaError_t gradients(morea_mlp *n, int b, const float *x, const float *t, cudaStream_t st)
{
    cudaError_t e = forward(n, b, x, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->loss, 0, sizeof(float), st);
    if (e == cudaSuccess) e = mlp_loss(b, n->n_out, n->Y, t, n->dY, n->loss, st);
    if (e == cudaSuccess)
        e = mlp_out_grads(b, n->h2, n->n_out, n->dY, n->H2, n->h2, n->W3b, n->h2, n->g + n->oW3, n->g + n->ob3,
                          n->dH2, n->h2, st);
    if (e == cudaSuccess) e = mlp_colsum(b, n->h2, n->dH2, n->h2, n->g + n->ob2, st);
    // dW2 = dH2^T H1  (K = batch, zero-padded to bpad)
    if (e == cudaSuccess) e = mlp_transpose(b, n->h2, n->bpad, n->dH2, n->h2, n->dH2T, n->bpad, st);
    if (e == cudaSuccess) e = mlp_transpose(b, n->h1, n->bpad, n->H1, n->h1, n->H1T, n->bpad, st);
    if (e == cudaSuccess)
        e = mlp_gemm_nt(n->h2, n->h1, n->bpad, n->dH2T, n->bpad, n->H1T, n->bpad, nullptr, nullptr, 0, 0,
                        n->g + n->oW2, n->h1, nullptr, 0, n->ws, n->ws_floats, n->status, st);
    // dH1 = (dH2 W2) [H1 > 0]
    if (e == cudaSuccess)
        e = mlp_gemm_nt(b, n->h1, n->h2, n->dH2, n->h2, n->W2Tb, n->h2, nullptr, n->H1, n->h1, 0, nullptr, 0, n->dH1,
                        n->h1, n->ws, n->ws_floats, n->status, st);
    if (e == cudaSuccess) e = mlp_colsum(b, n->h1, n->dH1, n->h1, n->g + n->ob1, st);
    // dW1 = dH1^T X
    if (e == cudaSuccess) e = mlp_transpose(b, n->h1, n->bpad, n->dH1, n->h1, n->dH1T, n->bpad, st);
    if (e == cudaSuccess) e = mlp_transpose(b, n->kin, n->bpad, n->X, n->kin, n->XT, n->bpad, st);
    if (e == cudaSuccess)
        e = mlp_gemm_nt(n->h1, n->kin, n->bpad, n->dH1T, n->bpad, n->XT, n->bpad, nullptr, nullptr, 0, 0,
                        n->g + n->oW1, n->kin, nullptr, 0, n->ws, n->ws_floats, n->status, st);
    return e;
}

}  // namespace

extern "C" {

morea_status morea_mlp_destroy(morea_mlp *n)
{
    if (!n) return MOREA_OK;
    DeviceGuard g(n->device);
    cudaError_t first = cudaSuccess;
    for (void *p : n->allocs) {
        cudaError_t e = cudaFree(p);
        if (first == cudaSuccess) first = e;
    }
    delete n;
    return from_cuda(first);
}

morea_status morea_mlp_create(int32_t n_in, int32_t h1, int32_t h2, int32_t n_out, int32_t max_batch,
                              morea_mlp **out)
{
    if (!out) return MOREA_EINVAL;
    *out = nullptr;
    if (n_in < 1 || h1 < 64 || h2 < 64 || h1 % 64 || h2 % 64 || n_out < 1 || n_out > 32 || max_batch < 1 ||
        (long long)n_in * max_batch > (1LL << 31) || (long long)h1 * up(n_in, 64) > (1LL << 31))
        return MOREA_EINVAL;
    morea_mlp *n = new (std::nothrow) morea_mlp();
    if (!n) return MOREA_ENOMEM;
    cudaGetDevice(&n->device);
    n->n_in = n_in;
    n->h1 = h1;
    n->h2 = h2;
    n->n_out = n_out;
    n->max_batch = max_batch;
    n->kin = (int)up(n_in, 64);
    n->bpad = (int)up(max_batch, 32);
    n->oW1 = 0;
    n->ob1 = n->oW1 + (long long)h1 * n->kin;
    n->oW2 = n->ob1 + h1;
    n->ob2 = n->oW2 + (long long)h2 * h1;
    n->oW3 = n->ob2 + h2;
    n->ob3 = n->oW3 + (long long)n_out * h2;
    n->n_params = n->ob3 + n_out;
    const size_t P = (size_t)n->n_params, B = (size_t)max_batch, BP = (size_t)n->bpad, bf = 2;
    cudaError_t e = dalloc(n, &n->w, P);
    if (e == cudaSuccess) e = dalloc(n, &n->g, P);
    if (e == cudaSuccess) e = dalloc(n, &n->m, P);
    if (e == cudaSuccess) e = dalloc(n, &n->v, P);
    unsigned char *p = nullptr;
    auto bfalloc = [&](void **dst, size_t elems) {
        if (e == cudaSuccess) {
            e = dalloc(n, &p, elems * bf);
            *dst = p;
        }
    };
    bfalloc(&n->W1b, (size_t)h1 * n->kin);
    bfalloc(&n->W2b, (size_t)h2 * h1);
    bfalloc(&n->W2Tb, (size_t)h1 * h2);
    bfalloc(&n->W3b, (size_t)n_out * h2);
    bfalloc(&n->X, B * n->kin);
    bfalloc(&n->XT, (size_t)n->kin * BP);
    bfalloc(&n->H1, B * h1);
    bfalloc(&n->H1T, (size_t)h1 * BP);
    bfalloc(&n->H2, B * h2);
    bfalloc(&n->dH2, B * h2);
    bfalloc(&n->dH2T, (size_t)h2 * BP);
    bfalloc(&n->dH1, B * h1);
    bfalloc(&n->dH1T, (size_t)h1 * BP);
    if (e == cudaSuccess) e = dalloc(n, &n->Y, B * n_out);
    if (e == cudaSuccess) e = dalloc(n, &n->dY, B * n_out);
    if (e == cudaSuccess) e = dalloc(n, &n->loss, 1);
    if (e == cudaSuccess) e = dalloc(n, &n->status, 1);
    n->ws_floats = 8LL * std::max(max_batch, h2) * h1;
    if (e == cudaSuccess) e = dalloc(n, &n->ws, (size_t)n->ws_floats);
    if (e == cudaSuccess) e = cudaMemset(n->status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(n->w, 0, P * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, P * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, P * sizeof(float));
    if (e == cudaSuccess) e = refresh_bf16(n, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        morea_mlp_destroy(n);
        return e == cudaErrorMemoryAllocation ? MOREA_ENOMEM : MOREA_ECUDA;
    }
    *out = n;
    return MOREA_OK;
}

morea_status morea_mlp_info(const morea_mlp *n, int64_t *n_params, int32_t *padded_inputs)
{
    if (!n) return MOREA_EINVAL;
    if (n_params) *n_params = n->n_params;
    if (padded_inputs) *padded_inputs = n->kin;
    return MOREA_OK;
}

morea_status morea_mlp_device_status(morea_mlp *n, uint32_t *bits, void *stream)
{
    if (!n || !bits) return MOREA_EINVAL;
    DeviceGuard g(n->device);
    cudaStream_t st = (cudaStream_t)stream;
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, n->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    *bits = (uint32_t)v;
    return from_cuda(e);
}

morea_status morea_mlp_set_params(morea_mlp *n, const float *params, void *stream)
{
    if (!n || !params) return MOREA_EINVAL;
    DeviceGuard g(n->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(n->w, params, sizeof(float) * n->n_params, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, sizeof(float) * n->n_params, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, sizeof(float) * n->n_params, st);
    if (e == cudaSuccess) e = refresh_bf16(n, st);
    n->step = 0;
    return from_cuda(e);
}

morea_status morea_mlp_get_params(morea_mlp *n, float *params, void *stream)
{
    if (!n || !params) return MOREA_EINVAL;
    DeviceGuard g(n->device);
    return from_cuda(cudaMemcpyAsync(params, n->w, sizeof(float) * n->n_params, cudaMemcpyDefault,
                                     (cudaStream_t)stream));
}

morea_status morea_mlp_forward(morea_mlp *n, int32_t batch, const float *x, float *y, void *stream)
{
    if (!n || !x || !y || batch < 1 || batch > n->max_batch) return MOREA_EINVAL;
    DeviceGuard g(n->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = forward(n, batch, x, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(y, n->Y, sizeof(float) * batch * n->n_out, cudaMemcpyDeviceToDevice, st);
    return from_cuda(e);
}

morea_status morea_mlp_gradients(morea_mlp *n, int32_t batch, const float *x, const float *t, float *grads,
                                 float *loss, void *stream)
{
    if (!n || !x || !t || batch < 1 || batch > n->max_batch) return MOREA_EINVAL;
    DeviceGuard g(n->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = gradients(n, batch, x, t, st);
    if (e == cudaSuccess && grads)
        e = cudaMemcpyAsync(grads, n->g, sizeof(float) * n->n_params, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, st);
    return from_cuda(e);
}

morea_status morea_mlp_train_step(morea_mlp *n, int32_t batch, const float *x, const float *t, float lr,
                                  float *loss, void *stream)
{
    if (!n || !x || !t || batch < 1 || batch > n->max_batch || !(lr > 0.0f)) return MOREA_EINVAL;
    DeviceGuard g(n->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = gradients(n, batch, x, t, st);
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - (float)std::pow((double)b1, (double)n->step);
    const float c2 = 1.0f - (float)std::pow((double)b2, (double)n->step);
    if (e == cudaSuccess) e = mlp_adam(n->n_params, n->w, n->g, n->m, n->v, lr, b1, b2, 1e-8f, c1, c2, nullptr, st);
    if (e == cudaSuccess) e = refresh_bf16(n, st);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, st);
    return from_cuda(e);
}

}  // extern "C"
