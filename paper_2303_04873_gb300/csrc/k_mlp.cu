// Surrogate network (step a10): a 3-layer perceptron n_in -> h1 -> h2 -> n_out
// over the per-vertex displacements of a solution, with BF16 weights and
// activations on the tensor cores and FP32 accumulation, trained on the GPU by
// these kernels (forward, backward, Adam).
//
// Every dense product is written as C[M x N] = A[M x K] . B[N x K]^T with both
// operands K-contiguous (the mma "row.col" form); transposes give the other
// layouts.  K dimensions are padded with zeros to a multiple of 64 (features)
// or 32 (batch), so the tiles never need a K bound check.
#include <cuda_bf16.h>

#include "morea_internal.cuh"
#include "morea_mlp.h"

namespace morea {

namespace {

using bf16 = __nv_bfloat16;

constexpr int GBM = 128, GBN = 128, GBK = 32, GPAD = 8;
constexpr int GSTR = GBK + GPAD;      // smem row stride in elements (80 bytes)

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid)
{
    const int bytes = valid ? 16 : 0;     // 0: zero-fill without reading
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem), "r"(bytes));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

__device__ __forceinline__ void ldsm_x4(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3, const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float *c, const unsigned *a, unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C = act(A . B^T + bias) (M x N), optionally masked by relu'(H) = [H > 0].
// Tiles 128 x 128 x 32, 8 warps as 2 (M) x 4 (N), warp tile 64 x 32.
__global__ void __launch_bounds__(256) k_gemm_nt(int M, int N, int K, const bf16 *__restrict__ A, int lda,
                                                 const bf16 *__restrict__ B, int ldb, const float *__restrict__ bias,
                                                 const bf16 *__restrict__ mask, int ldm, int relu, float *__restrict__ C,
                                                 int ldc, bf16 *__restrict__ Cb, int ldcb)
{
    __shared__ __align__(16) bf16 As[2][GBM][GSTR];
    __shared__ __align__(16) bf16 Bs[2][GBN][GSTR];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;

    auto load_tile = [&](int buf, int k0) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int chunk = tid + c * 256;          // 512 chunks of 16 B per operand tile
            const int r = chunk >> 2, kk = (chunk & 3) * 8;
            const int ga = min(m0 + r, M - 1), gb = min(n0 + r, N - 1);
            cp_async16(&As[buf][r][kk], A + (size_t)ga * lda + k0 + kk, m0 + r < M);
            cp_async16(&Bs[buf][r][kk], B + (size_t)gb * ldb + k0 + kk, n0 + r < N);
        }
        cp_async_commit();
    };

    const int nk = K / GBK;
    load_tile(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) {
            load_tile(buf ^ 1, (kt + 1) * GBK);
            cp_async_wait1();
        } else {
            cp_async_wait0();
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GBK; ks += 16) {
            unsigned af[4][4], bfr[2][4];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
                ldsm_x4(af[mi][0], af[mi][1], af[mi][2], af[mi][3],
                        &As[buf][wm + mi * 16 + (lane & 15)][ks + (lane >> 4) * 8]);
#pragma unroll
            for (int nj = 0; nj < 2; ++nj)
                ldsm_x4(bfr[nj][0], bfr[nj][1], bfr[nj][2], bfr[nj][3],
                        &Bs[buf][wn + nj * 16 + (lane >> 4) * 8 + (lane & 7)][ks + ((lane >> 3) & 1) * 8]);
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
                    mma_bf16(acc[mi][ni], af[mi], bfr[ni >> 1][(ni & 1) * 2], bfr[ni >> 1][(ni & 1) * 2 + 1]);
        }
        __syncthreads();
    }
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = m0 + wm + mi * 16 + g + h * 8;
                if (m >= M) continue;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int n = n0 + wn + ni * 8 + 2 * t + q;
                    if (n >= N) continue;
                    float v = acc[mi][ni][h * 2 + q];
                    if (bias) v += bias[n];
                    if (relu) v = fmaxf(v, 0.0f);
                    if (mask && !(__bfloat162float(mask[(size_t)m * ldm + n]) > 0.0f)) v = 0.0f;
                    if (C) C[(size_t)m * ldc + n] = v;
                    if (Cb) Cb[(size_t)m * ldcb + n] = __float2bfloat16(v);
                }
            }
}

// FP32 [rows][cols] -> BF16 [rows][ld] with zero padding up to ld (and rows up to rows_pad).
__global__ void k_to_bf16(int rows, int cols, int rows_pad, int ld, const float *__restrict__ x, bf16 *__restrict__ y)
{
    const long long total = (long long)rows_pad * ld;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / ld), c = (int)(i - (long long)r * ld);
        y[i] = __float2bfloat16(r < rows && c < cols ? x[(size_t)r * cols + c] : 0.0f);
    }
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

// dW3[o][k] = sum_b dY[b][o] H2[b][k];  db3[o] = sum_b dY[b][o]
__global__ void k_out_wgrad(int n, int h2, int n_out, const float *__restrict__ dY, const bf16 *__restrict__ H2, int ldh,
                            float *__restrict__ dW3, int ldw, float *__restrict__ db3)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_out * h2) {
        const int o = i / h2, k = i - o * h2;
        float s = 0.0f;
        for (int b = 0; b < n; ++b) s = fmaf(dY[(size_t)b * n_out + o], __bfloat162float(H2[(size_t)b * ldh + k]), s);
        dW3[(size_t)o * ldw + k] = s;
    } else if (i < n_out * h2 + n_out) {
        const int o = i - n_out * h2;
        float s = 0.0f;
        for (int b = 0; b < n; ++b) s += dY[(size_t)b * n_out + o];
        db3[o] = s;
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

// db[c] = sum_r D[r][c]  (column sums of a BF16 matrix, FP32)
__global__ void k_colsum(int rows, int cols, const bf16 *__restrict__ D, int ld, float *__restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.0f;
    for (int r = 0; r < rows; ++r) s += __bfloat162float(D[(size_t)r * ld + c]);
    out[c] = s;
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

cudaError_t mlp_gemm_nt(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias,
                        const void *mask, int ldm, int relu, float *C, int ldc, void *Cb, int ldcb, cudaStream_t st)
{
    dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
    k_gemm_nt<<<grid, 256, 0, st>>>(M, N, K, (const bf16 *)A, lda, (const bf16 *)B, ldb, bias, (const bf16 *)mask, ldm,
                                    relu, C, ldc, (bf16 *)Cb, ldcb);
    return cudaGetLastError();
}

cudaError_t mlp_to_bf16(int rows, int cols, int rows_pad, int ld, const float *x, void *y, cudaStream_t st)
{
    k_to_bf16<<<g1d((long long)rows_pad * ld), 256, 0, st>>>(rows, cols, rows_pad, ld, x, (bf16 *)y);
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
    k_out_wgrad<<<(n_out * h2 + n_out + 255) / 256, 256, 0, st>>>(n, h2, n_out, dY, (const bf16 *)H2, ldh, dW3, h2, db3);
    k_out_bgrad<<<g1d((long long)n * h2), 256, 0, st>>>(n, h2, n_out, dY, (const bf16 *)W3, ldw, (const bf16 *)H2, ldh,
                                                         (bf16 *)dH2, ldd);
    return cudaGetLastError();
}

cudaError_t mlp_colsum(int rows, int cols, const void *D, int ld, float *out, cudaStream_t st)
{
    k_colsum<<<(cols + 255) / 256, 256, 0, st>>>(rows, cols, (const bf16 *)D, ld, out);
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
