// Launchers of the surrogate-network kernels (k_mlp.cu).  Internal.
#pragma once

#include <cuda_runtime.h>

namespace morea {

// C = act(A . B^T + bias) on the tcgen05 tensor cores (k_gemm_tc.cu):
// A [M][K], B [N][K] BF16, 16-byte aligned, lda/ldb multiples of 8; optional
// ReLU, optional mask [H > 0] (BF16 H), FP32 output C and/or BF16 output Cb.
// A wait that gives up inside the kernel sets bit 0 of *status (device).
// ws (ws_floats FP32, may be NULL) is the split-K workspace: products with
// few output tiles and a long K are split over up to 8 CTAs per tile.
cudaError_t mlp_gemm_nt(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias,
                        const void *mask, int ldm, int relu, float *C, int ldc, void *Cb, int ldcb, float *ws,
                        long long ws_floats, int *status, cudaStream_t st);
int mlp_gemm_splits(int M, int N, int K);
cudaError_t mlp_to_bf16(int rows, int cols, int rows_pad, int ld, const float *x, void *y, cudaStream_t st);
cudaError_t mlp_transpose(int rows, int cols, int rows_pad, const void *in, int ldi, void *out, int ldo, cudaStream_t st);
cudaError_t mlp_out_fwd(int n, int h2, int n_out, const void *H2, int ldh, const void *W3, int ldw, const float *b3,
                        float *Y, cudaStream_t st);
cudaError_t mlp_loss(int n, int n_out, const float *Y, const float *T, float *dY, float *loss, cudaStream_t st);
cudaError_t mlp_out_grads(int n, int h2, int n_out, const float *dY, const void *H2, int ldh, const void *W3, int ldw,
                          float *dW3, float *db3, void *dH2, int ldd, cudaStream_t st);
cudaError_t mlp_colsum(int rows, int cols, const void *D, int ld, float *out, cudaStream_t st);
cudaError_t mlp_adam(long long n, float *w, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                     float c1, float c2, void *wb, cudaStream_t st);
cudaError_t mlp_cast(long long n, const float *w, void *wb, cudaStream_t st);

}  // namespace morea
