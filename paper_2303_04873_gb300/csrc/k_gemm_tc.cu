// Dense products of the surrogate network (step a10) on the 5th-generation
// tensor cores: C[M x N] = A[M x K] . B[N x K]^T, both operands BF16 and
// K-contiguous, FP32 accumulation in tensor memory.
//
// One CTA computes one 128 x 128 tile of C with three roles:
//   warp 0 (one lane)  TMA producer: 128 x 64 tiles of A and B into a 6-stage
//                      shared-memory ring (128-byte swizzle), completion on
//                      the stage's "full" mbarrier;
//   warp 1             allocates 128 TMEM columns; one lane issues four
//                      tcgen05.mma (128 x 128 x 16, kind::f16) per stage and
//                      commits them to the stage's "empty" mbarrier, and the
//                      whole tile to "done";
//   warps 2-5          epilogue: each reads its 32 TMEM lanes (rows) with
//                      tcgen05.ld, adds the bias, applies ReLU / the ReLU'
//                      mask, and stores FP32 and/or BF16.
// Rows and columns past M, N and K are zero-filled by TMA and not stored.
// Split K: with gridDim.z = S > 1, CTA z takes k-blocks [z nk / S, (z+1) nk / S)
// and stores its raw FP32 tile into ws[z][M][N]; k_splitk_reduce then sums
// the S partial tiles in order and applies the epilogue.
// Every mbarrier wait is bounded: on timeout the CTA sets *status, waits
// (bounded) for its own copies in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "morea_internal.cuh"
#include "morea_mlp.h"

namespace morea {

namespace {

using bf16 = __nv_bfloat16;

constexpr int TBM = 128, TBN = 128, TBK = 64, TST = 6;
constexpr int kTileA = TBM * TBK * 2;                  // 16 KB
constexpr int kTileB = TBN * TBK * 2;                  // 16 KB
constexpr int kStage = kTileA + kTileB;
constexpr uint32_t kTmemCols = 128;                    // FP32 accumulator 128 lanes x 128 columns
constexpr int kSmemBytes = TST * kStage + 256 + 1024;  // ring + barriers + alignment slack
constexpr long long kSpinLimit = 1LL << 24;            // try_wait polls before a wait gives up

// Instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1),
// A and B BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                            ((uint32_t)(TBM >> 4) << 24);

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of the given parity to complete; false after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (long long i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with the 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes
// apart (stride byte offset), version 1 in bits 46-48, swizzle mode 2 in
// bits 61-63.  The start address moves 32 bytes per 16-element K step.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(192, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N, int K,
              const float *__restrict__ bias, const bf16 *__restrict__ mask, int ldm, int relu, float *__restrict__ C,
              int ldc, bf16 *__restrict__ Cb, int ldcb, float *__restrict__ ws, int *status)
{
    extern __shared__ uint8_t dsm[];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int cta_err;
    const uint32_t raw = saddr(dsm);
    const uint32_t base = (raw + 1023u) & ~1023u;       // the swizzle pattern is anchored at 1024 B
    const uint32_t bar0 = base + TST * kStage;
    const uint32_t done = bar0 + 8u * (2 * TST);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
    const int nk_all = (K + TBK - 1) / TBK;
    const int kb0 = (int)(((long long)blockIdx.z * nk_all) / gridDim.z);
    const int nk = (int)(((long long)(blockIdx.z + 1) * nk_all) / gridDim.z) - kb0;
    if (gridDim.z > 1) {            // this CTA's share of K: raw partial tile, no epilogue
        C = ws + (size_t)blockIdx.z * M * N;
        ldc = N;
        Cb = nullptr;
        bias = nullptr;
        mask = nullptr;
        relu = 0;
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < TST; ++s) {
            mbar_init(bar0 + 8u * s, 1);                  // full[s]: producer arrive + TMA bytes
            mbar_init(bar0 + 8u * (TST + s), 1);          // empty[s]: MMA commit
        }
        mbar_init(done, 1);
        cta_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % TST;
                if (kb >= TST && !mbar_wait(bar0 + 8u * (TST + s), ((kb / TST) - 1) & 1)) {
                    cta_err = 1;
                    break;
                }
                const uint32_t dst = base + s * kStage;
                mbar_expect_tx(bar0 + 8u * s, kStage);
                tma_load_2d(dst, &ta, bar0 + 8u * s, (kb0 + kb) * TBK, m0);
                tma_load_2d(dst + kTileA, &tb, bar0 + 8u * s, (kb0 + kb) * TBK, n0);
                ++issued;
            }
            if (cta_err) {   // let the copies in flight land before the CTA exits
                for (int kb = issued > TST ? issued - TST : 0; kb < issued; ++kb)
                    mbar_wait(bar0 + 8u * (kb % TST), (kb / TST) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % TST;
                if (!mbar_wait(bar0 + 8u * s, (kb / TST) & 1)) {
                    cta_err = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t a = base + s * kStage, b = a + kTileA;
#pragma unroll
                for (int k = 0; k < TBK / 16; ++k)
                    umma_bf16(tmem, sw128_desc(a + 32u * k), sw128_desc(b + 32u * k), (kb | k) != 0 ? 1u : 0u);
                umma_commit(bar0 + 8u * (TST + s));      // stage s may be refilled once these have read it
            }
            umma_commit(done);                           // all MMAs issued by this thread
        }
    } else {
        const int q = warp & 3;                          // TMEM lanes 32q .. 32q + 31
        const bool ok = mbar_wait(done, 0);
        tc_fence_after();
        if (!ok) cta_err = 1;
        if (ok && !cta_err) {
            const int m = m0 + 32 * q + lane;
            // 16 consecutive columns per thread: vector loads and stores when
            // the chunk is inside N and the row offsets keep 16-byte alignment
            const bool vec_c = C && (ldc % 4) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0;
            const bool vec_b = Cb && (ldcb % 8) == 0 && (reinterpret_cast<uintptr_t>(Cb) & 15) == 0;
            const bool vec_m = mask && (ldm % 8) == 0 && (reinterpret_cast<uintptr_t>(mask) & 15) == 0;
#pragma unroll 1
            for (int c0 = 0; c0 < TBN; c0 += 16) {
                uint32_t r[16];
                __syncwarp();                            // tcgen05.ld is warp-collective
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, r);
                const int nb = n0 + c0;
                if (m >= M || nb >= N) continue;
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    v[j] = __uint_as_float(r[j]);
                    if (bias && nb + j < N) v[j] += __ldg(bias + nb + j);
                    if (relu) v[j] = fmaxf(v[j], 0.0f);
                }
                const bool full = nb + 16 <= N;
                if (mask) {
                    const bf16 *mp = mask + (size_t)m * ldm + nb;
                    if (full && vec_m) {
                        const uint4 w0 = *reinterpret_cast<const uint4 *>(mp);
                        const uint4 w1 = *reinterpret_cast<const uint4 *>(mp + 8);
                        const bf16 *h0 = reinterpret_cast<const bf16 *>(&w0), *h1 = reinterpret_cast<const bf16 *>(&w1);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            if (!(__bfloat162float(h0[j]) > 0.0f)) v[j] = 0.0f;
                            if (!(__bfloat162float(h1[j]) > 0.0f)) v[j + 8] = 0.0f;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (nb + j < N && !(__bfloat162float(mp[j]) > 0.0f)) v[j] = 0.0f;
                    }
                }
                if (C) {
                    float *cp = C + (size_t)m * ldc + nb;
                    if (full && vec_c) {
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            *reinterpret_cast<float4 *>(cp + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (nb + j < N) cp[j] = v[j];
                    }
                }
                if (Cb) {
                    bf16 *bp = Cb + (size_t)m * ldcb + nb;
                    if (full && vec_b) {
                        uint4 w[2];
                        __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(w);
#pragma unroll
                        for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                        *reinterpret_cast<uint4 *>(bp) = w[0];
                        *reinterpret_cast<uint4 *>(bp + 8) = w[1];
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (nb + j < N) bp[j] = __float2bfloat16(v[j]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
    if (threadIdx.x == 0 && cta_err) atomicOr(status, 1);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// [rows][cols] BF16 matrix with row stride ld (elements), read in 128 x 64 boxes.
cudaError_t make_map(CUtensorMap *map, const void *ptr, int cols, int rows, int ld)
{
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    if ((reinterpret_cast<uintptr_t>(ptr) & 15) || (ld % 8) || cols > ld || rows < 1 || cols < 1)
        return cudaErrorInvalidValue;
    const cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TBK, (cuuint32_t)TBM};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), gdim, gstride, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Sum of the split-K partial tiles in split order, then the epilogue.
__global__ void k_splitk_reduce(int M, int N, int splits, const float *__restrict__ ws, const float *__restrict__ bias,
                                const bf16 *__restrict__ mask, int ldm, int relu, float *__restrict__ C, int ldc,
                                bf16 *__restrict__ Cb, int ldcb)
{
    const long long total = (long long)M * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(i / N), n = (int)(i - (long long)m * N);
        float v = 0.0f;
        for (int z = 0; z < splits; ++z) v += ws[(size_t)z * total + i];
        if (bias) v += bias[n];
        if (relu) v = fmaxf(v, 0.0f);
        if (mask && !(__bfloat162float(mask[(size_t)m * ldm + n]) > 0.0f)) v = 0.0f;
        if (C) C[(size_t)m * ldc + n] = v;
        if (Cb) Cb[(size_t)m * ldcb + n] = __float2bfloat16(v);
    }
}

}  // namespace

int mlp_gemm_splits(int M, int N, int K)
{
    const long long tiles = (long long)((M + TBM - 1) / TBM) * ((N + TBN - 1) / TBN);
    const int nk = (K + TBK - 1) / TBK;
    // enough CTAs to cover the SMs, at least 2 k-blocks each, at most 8 splits
    // (one CTA streams its operands through TMA at a bounded rate, so short
    // products gain from more CTAs even at the cost of the ordered reduction)
    long long s = std::min<long long>(nk / 2, (148 + tiles - 1) / tiles);
    return (int)std::max<long long>(1, std::min<long long>(s, 8));
}

cudaError_t mlp_gemm_nt(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias,
                        const void *mask, int ldm, int relu, float *C, int ldc, void *Cb, int ldcb, float *ws,
                        long long ws_floats, int *status, cudaStream_t st)
{
    if (M < 1 || N < 1 || K < 1) return cudaErrorInvalidValue;
    CUtensorMap ta, tb;
    cudaError_t e = make_map(&ta, A, K, M, lda);
    if (e == cudaSuccess) e = make_map(&tb, B, K, N, ldb);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    int splits = ws ? mlp_gemm_splits(M, N, K) : 1;
    while (splits > 1 && (long long)splits * M * N > ws_floats) --splits;
    const dim3 grid((N + TBN - 1) / TBN, (M + TBM - 1) / TBM, splits);
    k_gemm_tc<<<grid, 192, kSmemBytes, st>>>(ta, tb, M, N, K, bias, (const bf16 *)mask, ldm, relu, C, ldc,
                                            (bf16 *)Cb, ldcb, ws, status);
    e = cudaGetLastError();
    if (e != cudaSuccess || splits == 1) return e;
    const long long total = (long long)M * N;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
    k_splitk_reduce<<<blocks, 256, 0, st>>>(M, N, splits, ws, bias, (const bf16 *)mask, ldm, relu, C, ldc, (bf16 *)Cb,
                                           ldcb);
    return cudaGetLastError();
}

}  // namespace morea
