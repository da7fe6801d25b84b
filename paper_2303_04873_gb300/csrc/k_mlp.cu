// Surrogate network (step a10): a 3-layer perceptron n_in -> h1 -> h2 -> n_out
// over the per-vertex displacements of a solution, with BF16 weights and
// activations and FP32 accumulation, trained on the GPU by these kernels
// (forward, backward, Adam).  The dense products C = A . B^T, both operands
// K-contiguous, run on the tcgen05 tensor cores (k_gemm_tc.cu); this file
// holds the element-wise and small kernels around them.  Transposes give the
// K-contiguous layouts; K dimensions are padded with zeros to a multiple of
// 64 (features) or 32 (batch).
#include <cuda_bf16.h>

#include "morea_internal.cuh"
#include "morea_mlp.h"

namespace morea {

namespace {

using bf16 = __nv_bfloat16;

// FP32 [rows][cols] -> BF16 [rows][ld] with zero padding up to ld (and rows up to rows_pad).
__global__ void k_to_bf16(int r0, int rows, int cols, int ld, const float *__restrict__ x, bf16 *__restrict__ y)
{
    const int r = r0 + blockIdx.y;                     // one row per grid row, columns in 2-element steps
    const int c = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (c >= ld) return;
    const float *xr = x + (size_t)r * cols;
    const float a = r < rows && c < cols ? xr[c] : 0.0f;
    const float b = r < rows && c + 1 < cols ? xr[c + 1] : 0.0f;
    *reinterpret_cast<__nv_bfloat162 *>(y + (size_t)r * ld + c) = __floats2bfloat162_rn(a, b);
}

// out[c][r] = in[r][c] for r < rows (zero for rows <= r < rows_pad), c < cols.
__global__ void k_transpose(int rows, int cols, int rows_pad, const bf16 *__restrict__ in, int ldi,
                            bf16 *__restrict__ out, int ldo)
{
    __shared__ bf16 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? in[(size_t)r * ldi + c] : __float2bfloat16(0.0f);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows_pad) out[(size_t)c * ldo + r] = tile[threadIdx.x][i];
    }
}

// Output layer: Y[b][o] = sum_k H2[b][k] W3[o][k] + b3[o]  (FP32 accumulation).
__global__ void k_out_fwd(int n, int h2, int n_out, const bf16 *__restrict__ H2, int ldh, const bf16 *__restrict__ W3,
                          int ldw, const float *__restrict__ b3, float *__restrict__ Y)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n * n_out) return;
    const int b = warp / n_out, o = warp - b * n_out;
    float s = 0.0f;
    for (int k = lane; k < h2; k += 32)
        s = fmaf(__bfloat162float(H2[(size_t)b * ldh + k]), __bfloat162float(W3[(size_t)o * ldw + k]), s);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) Y[(size_t)b * n_out + o] = s + b3[o];
}

// MSE loss over n x n_out and dY = 2 (Y - T) / (n n_out).
__global__ void k_loss(int n, int n_out, const float *__restrict__ Y, const float *__restrict__ Tg, float *__restrict__ dY,
                       float *loss)
{
    __shared__ float sh[256];
    const int total = n * n_out;
    float s = 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const float d = Y[i] - Tg[i];
        dY[i] = 2.0f * d / (float)total;
        s += d * d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) atomicAdd(loss, sh[0] / (float)total);
}

// dW3[o][k] = sum_b dY[b][o] H2[b][k];  db3[o] = sum_b dY[b][o].
// Block (32 columns k, 32 row groups) per (column tile, o); the 32 partial
// sums are combined in a fixed order.
__global__ void k_out_wgrad(int n, int h2, int n_out, const float *__restrict__ dY, const bf16 *__restrict__ H2, int ldh,
                            float *__restrict__ dW3, int ldw, float *__restrict__ db3)
{
    __shared__ float part[32][33], pb[32];
    const int o = blockIdx.y, k = blockIdx.x * 32 + threadIdx.x;
    float s = 0.0f, sb = 0.0f;
    for (int b = threadIdx.y; b < n; b += 32) {
        const float d = dY[(size_t)b * n_out + o];
        if (k < h2) s = fmaf(d, __bfloat162float(H2[(size_t)b * ldh + k]), s);
        sb += d;
    }
    part[threadIdx.y][threadIdx.x] = s;
    if (threadIdx.x == 0) pb[threadIdx.y] = sb;
    __syncthreads();
    if (threadIdx.y == 0) {
        float t = 0.0f;
#pragma unroll
        for (int g = 0; g < 32; ++g) t += part[g][threadIdx.x];
        if (k < h2) dW3[(size_t)o * ldw + k] = t;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            float u = 0.0f;
#pragma unroll
            for (int g = 0; g < 32; ++g) u += pb[g];
            db3[o] = u;
        }
    }
}

// dH2[b][k] = (sum_o dY[b][o] W3[o][k]) [H2[b][k] > 0]  (BF16)
__global__ void k_out_bgrad(int n, int h2, int n_out, const float *__restrict__ dY, const bf16 *__restrict__ W3, int ldw,
                            const bf16 *__restrict__ H2, int ldh, bf16 *__restrict__ dH2, int ldd)
{
    const long long total = (long long)n * h2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / h2), k = (int)(i - (long long)b * h2);
        float s = 0.0f;
        for (int o = 0; o < n_out; ++o) s = fmaf(dY[(size_t)b * n_out + o], __bfloat162float(W3[(size_t)o * ldw + k]), s);
        if (!(__bfloat162float(H2[(size_t)b * ldh + k]) > 0.0f)) s = 0.0f;
        dH2[(size_t)b * ldd + k] = __float2bfloat16(s);
    }
}

// db[c] = sum_r D[r][c]  (column sums of a BF16 matrix, FP32): 32 columns
// per block, 32 row groups combined in a fixed order.
__global__ void k_colsum(int rows, int cols, const bf16 *__restrict__ D, int ld, float *__restrict__ out)
{
    __shared__ float part[32][33];
    const int c = blockIdx.x * 32 + threadIdx.x;
    float s = 0.0f;
    if (c < cols)
        for (int r = threadIdx.y; r < rows; r += 32) s += __bfloat162float(D[(size_t)r * ld + c]);
    part[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && c < cols) {
        float t = 0.0f;
#pragma unroll
        for (int g = 0; g < 32; ++g) t += part[g][threadIdx.x];
        out[c] = t;
    }
}

// Adam on the FP32 master parameters, then the BF16 working copy.
__global__ void k_adam(long long n, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                       bf16 *__restrict__ wb)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16(wi);
    }
}

__global__ void k_cast(long long n, const float *__restrict__ w, bf16 *__restrict__ wb)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        wb[i] = __float2bfloat16(w[i]);
}

inline int g1d(long long work) { return (int)std::max<long long>(1, std::min<long long>((work + 255) / 256, 4096)); }

}  // namespace

cudaError_t mlp_to_bf16(int rows, int cols, int rows_pad, int ld, const float *x, void *y, cudaStream_t st)
{
    if (ld % 2) return cudaErrorInvalidValue;
    for (int r0 = 0; r0 < rows_pad; r0 += 65535)
        k_to_bf16<<<dim3((ld / 2 + 255) / 256, std::min(65535, rows_pad - r0)), 256, 0, st>>>(r0, rows, cols, ld, x,
                                                                                            (bf16 *)y);
    return cudaGetLastError();
}

cudaError_t mlp_transpose(int rows, int cols, int rows_pad, const void *in, int ldi, void *out, int ldo, cudaStream_t st)
{
    dim3 grid((cols + 31) / 32, (rows_pad + 31) / 32);
    k_transpose<<<grid, dim3(32, 8), 0, st>>>(rows, cols, rows_pad, (const bf16 *)in, ldi, (bf16 *)out, ldo);
    return cudaGetLastError();
}

cudaError_t mlp_out_fwd(int n, int h2, int n_out, const void *H2, int ldh, const void *W3, int ldw, const float *b3,
                        float *Y, cudaStream_t st)
{
    const long long warps = (long long)n * n_out;
    k_out_fwd<<<(int)((warps * 32 + 255) / 256), 256, 0, st>>>(n, h2, n_out, (const bf16 *)H2, ldh, (const bf16 *)W3,
                                                              ldw, b3, Y);
    return cudaGetLastError();
}

cudaError_t mlp_loss(int n, int n_out, const float *Y, const float *T, float *dY, float *loss, cudaStream_t st)
{
    k_loss<<<g1d((long long)n * n_out), 256, 0, st>>>(n, n_out, Y, T, dY, loss);
    return cudaGetLastError();
}

cudaError_t mlp_out_grads(int n, int h2, int n_out, const float *dY, const void *H2, int ldh, const void *W3, int ldw,
                          float *dW3, float *db3, void *dH2, int ldd, cudaStream_t st)
{
    k_out_wgrad<<<dim3((h2 + 31) / 32, n_out), dim3(32, 32), 0, st>>>(n, h2, n_out, dY, (const bf16 *)H2, ldh, dW3, h2,
                                                                    db3);
    k_out_bgrad<<<g1d((long long)n * h2), 256, 0, st>>>(n, h2, n_out, dY, (const bf16 *)W3, ldw, (const bf16 *)H2, ldh,
                                                         (bf16 *)dH2, ldd);
    return cudaGetLastError();
}

cudaError_t mlp_colsum(int rows, int cols, const void *D, int ld, float *out, cudaStream_t st)
{
    k_colsum<<<(cols + 31) / 32, dim3(32, 32), 0, st>>>(rows, cols, (const bf16 *)D, ld, out);
    return cudaGetLastError();
}

cudaError_t mlp_adam(long long n, float *w, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                     float c1, float c2, void *wb, cudaStream_t st)
{
    k_adam<<<g1d(n), 256, 0, st>>>(n, w, g, m, v, lr, b1, b2, eps, c1, c2, (bf16 *)wb);
    return cudaGetLastError();
}

cudaError_t mlp_cast(long long n, const float *w, void *wb, cudaStream_t st)
{
    k_cast<<<g1d(n), 256, 0, st>>>(n, w, (bf16 *)wb);
    return cudaGetLastError();
}

}  // namespace morea
