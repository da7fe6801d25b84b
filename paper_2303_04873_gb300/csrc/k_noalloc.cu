// Allocation-free variant of the tet pass: fold constraint and deformation
// magnitude of a batch of solutions without a problem handle.
//
// Who needs this: code that runs where cudaMalloc is not available or not
// allowed -- for example a caller that is itself inside another library's
// allocator or memory pool and must not re-enter it, or an environment that
// only gives out pre-sized device buffers.  Such a caller can still hand in
// its own input and output buffers; the per-(solution, tet) intermediate
// values, which the handle-based path keeps in memory allocated by
// morea_create_problem, live here in one fixed file-scope device array.
//
// That array is part of the library's device image, so every GPU that loads
// the library holds it until the process exits.  All calls on a device share
// it: two calls whose work overlaps on the GPU (different streams, no
// ordering between them) race on it.  Calls on one stream are ordered and
// safe.  Every slot the reduction reads is written earlier in the same call,
// so nothing in the array needs clearing between calls.
#include <algorithm>
#include <mutex>

#include "morea_device.cuh"

namespace morea {

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)MOREA_NOALLOC_MAX_TET_EVALS * sizeof(TetOut);

// The scratch: per (solution, tet) fold flags, integer severity and magnitude.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device.  In host code g_noalloc_scratch names a host-side shadow, not
// device memory, so the kernels get the address from cudaGetSymbolAddress.
// The address is cached for the life of the process: after cudaDeviceReset
// on a device the cached value is stale, so the entry point is not
// supported on that device after a reset.
cudaError_t noalloc_scratch(TetOut **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = (TetOut *)g_noalloc_addr[dev];
    return cudaSuccess;
}

__global__ void __launch_bounds__(kBlock) k_tet_noalloc(DevProblem P, int n_sol, const int *__restrict__ tets,
                                                       const float *__restrict__ ref, const float *__restrict__ src,
                                                       const float *__restrict__ tgt, TetOut *scratch)
{
    const int T = P.n_tets, V = P.n_points;
    const long long total = (long long)n_sol * T;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / T), t = (int)(e - (long long)i * T);
        int v[4] = {tets[4 * t], tets[4 * t + 1], tets[4 * t + 2], tets[4 * t + 3]};
        if (min(min(v[0], v[1]), min(v[2], v[3])) < 0 || max(max(v[0], v[1]), max(v[2], v[3])) >= V) {
            // a vertex id out of range: no read, the solution reports NaN / folded
            TetOut bad;
            bad.e_mag = __int_as_float(0x7fc00000);
            bad.folded = 3u;
            bad.sev = 0ull;
            scratch[e] = bad;
            continue;
        }
        // same orientation rule as problem creation: swap the last two
        // vertices of a tet whose reference volume is negative; a zero
        // reference volume (rejected at problem creation) gives NaN / folded
        int4 qr[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) qr[m] = snap3(ref + 3 * (size_t)v[m], P);
        const double dref = orient_d(qr[0], qr[1], qr[2], qr[3]);
        if (dref == 0.0) {
            TetOut bad;
            bad.e_mag = __int_as_float(0x7fc00000);
            bad.folded = 3u;
            bad.sev = 0ull;
            scratch[e] = bad;
            continue;
        }
        if (dref < 0.0) {
            const int tmp = v[2];
            v[2] = v[3];
            v[3] = tmp;
        }
        int4 qs[4], qt[4];
        const float *ps = src + (size_t)i * V * 3, *pt = tgt + (size_t)i * V * 3;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            qs[m] = snap3(ps + 3 * (size_t)v[m], P);
            qt[m] = snap3(pt + 3 * (size_t)v[m], P);
        }
        TetOut o;
        tet_terms(qs, qt, P, t, o);
        scratch[e] = o;
    }
}

template <typename T>
__device__ __forceinline__ T block_sum_na(T v, T *sh)
{
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
#pragma unroll
    for (int o = kBlock / 2; o > 0; o >>= 1) {
        if (tid < o) sh[tid] = sh[tid] + sh[tid + o];
        __syncthreads();
    }
    T r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kBlock) k_reduce_noalloc(int T, int S, const TetOut *__restrict__ scratch,
                                                          double *f_mag, uint8_t *folded, double *severity)
{
    __shared__ double shd[kBlock];
    __shared__ unsigned long long shu[kBlock];
    const int i = blockIdx.x;
    double mag = 0.0;
    unsigned long long nf = 0, sev = 0;
    for (int t = threadIdx.x; t < T; t += kBlock) {
        const TetOut o = scratch[(size_t)i * T + t];
        mag += (double)o.e_mag;
        nf += ((o.folded & 1u) != 0) + ((o.folded & 2u) != 0);
        sev += o.sev;
    }
    mag = block_sum_na<double>(mag, shd);
    nf = block_sum_na<unsigned long long>(nf, shu);
    sev = block_sum_na<unsigned long long>(sev, shu);
    if (threadIdx.x == 0) {
        f_mag[i] = mag / (10.0 * (double)T);
        folded[i] = nf > 0 ? 1 : 0;
        if (severity) {
            const double s = (double)S;
            severity[i] = (double)sev / (6.0 * s * s * s);
        }
    }
}

}  // namespace

}  // namespace morea

using namespace morea;

extern "C" morea_status morea_fold_magnitude_noalloc(int32_t n_sol, int32_t n_points, int32_t n_tets,
                                                     const int32_t *tets, const float *ref_points,
                                                     const float *cdelta, int32_t nx, int32_t ny, int32_t nz,
                                                     int32_t subvoxel_bits, const float *src_pts,
                                                     const float *tgt_pts, double *f_mag, uint8_t *folded,
                                                     double *severity, void *stream)
{
    if (n_sol < 1 || n_points < 4 || n_tets < 1 || !tets || !ref_points || !cdelta || !src_pts || !tgt_pts ||
        !f_mag || !folded)
        return MOREA_EINVAL;
    if (nx < 2 || ny < 2 || nz < 2) return MOREA_EINVAL;
    // the same grid as morea_create_problem: the box limit and the 64-bit
    // severity bound, with 0 picking the largest k <= 8 that meets both
    const int k = choose_subvoxel_bits(subvoxel_bits, nx, ny, nz, n_tets);
    if (k < 0) return MOREA_EINVAL;
    // the scratch holds MOREA_NOALLOC_MAX_TET_EVALS (solution, tet) records
    if ((long long)n_sol * n_tets > (long long)MOREA_NOALLOC_MAX_TET_EVALS) return MOREA_EINVAL;
    TetOut *scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) return MOREA_ECUDA;
    DevProblem P{};
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    P.kbits = k;
    P.S = 1 << k;
    P.H = 1 << (k - 1);
    P.n_points = n_points;
    P.n_tets = n_tets;
    P.cdelta = cdelta;
    cudaStream_t st = (cudaStream_t)stream;
    const long long work = (long long)n_sol * n_tets;
    const int grid = (int)std::max<long long>(1, std::min<long long>((work + kBlock - 1) / kBlock,
                                                                     (long long)sm_count() * 16));
    k_tet_noalloc<<<grid, kBlock, 0, st>>>(P, n_sol, tets, ref_points, src_pts, tgt_pts, scratch);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_reduce_noalloc<<<n_sol, kBlock, 0, st>>>(n_tets, P.S, scratch, f_mag, folded, severity);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? MOREA_OK : MOREA_ECUDA;
}
