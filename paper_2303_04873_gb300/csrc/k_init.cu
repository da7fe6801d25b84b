// Initialisation noise (Sec. 4.2.2, App. A.5; reading R18): Gaussian kernels
// placed on both images attract the mesh points in rounds.  A round moves
// every point x by sum_k a_k exp(-|c_k - x|^2 / (2 sigma_k^2)) (c_k - x) and
// is kept if no tet of the moved mesh is folded; the first round that folds
// ends the process for that mesh.
//
// One block per (solution, mesh).  The mesh stays in shared memory for all
// rounds: a round computes every point's candidate (threads over points,
// the kernel list in shared memory), then the exact orientation of every
// tet on the snapped candidates (threads over tets), and one block-wide OR
// decides.  Positions are FP64 with explicitly rounded operations and exp is
// evaluated by range reduction with ln 2 and a degree-13 Taylor series in
// Horner form, every step one rounded IEEE operation, so the positions
// equal the plain definition bit for bit.
#include "morea_device.cuh"

namespace morea {

namespace {

constexpr int kInitThreads = 256;

// exp(t) for t <= 0; zero below -64.  n = rint(t / ln2) lies in [-93, 0],
// so 2^n is a normal power of two and the final scaling is exact.
__device__ __forceinline__ double attraction_exp(double t)
{
    const double kLn2 = 0.6931471805599453;
    if (!(t >= -64.0)) return 0.0;
    const double n = rint(__ddiv_rn(t, kLn2));
    const double r = __dsub_rn(t, __dmul_rn(n, kLn2));
    double s = 1.0;
#pragma unroll
    for (int k = 13; k >= 1; --k) s = __dadd_rn(1.0, __ddiv_rn(__dmul_rn(r, s), (double)k));
    return __dmul_rn(s, __longlong_as_double((long long)(1023 + (int)n) << 52));
}

__global__ void __launch_bounds__(kInitThreads) k_init(const DevProblem *__restrict__ dp, float *src, float *tgt,
                                                       const uint8_t *__restrict__ fixed, int K,
                                                       const float *__restrict__ kernels, int max_rounds,
                                                       int *__restrict__ rounds_out)
{
    extern __shared__ float sm[];                // [5K] kernels, [3V] positions, [3V] candidates
    const DevProblem &P = *dp;
    const int V = P.n_points, T = P.n_tets;
    const int sol = blockIdx.x >> 1, mesh = blockIdx.x & 1;
    float *X = (mesh == 0 ? src : tgt) + (size_t)sol * V * 3;
    const float *kg = kernels + ((size_t)sol * 2 + mesh) * K * 5;
    float *ks = sm, *pos = sm + 5 * K, *cand = pos + 3 * V;
    for (int i = threadIdx.x; i < 5 * K; i += blockDim.x) ks[i] = kg[i];
    for (int i = threadIdx.x; i < 3 * V; i += blockDim.x) pos[i] = X[i];
    __syncthreads();
    int kept = 0;
    for (int round = 0; round < max_rounds; ++round) {
        for (int v = threadIdx.x; v < V; v += blockDim.x) {
            const double x0 = pos[3 * v], x1 = pos[3 * v + 1], x2 = pos[3 * v + 2];
            double d0 = 0.0, d1 = 0.0, d2 = 0.0;
            for (int k = 0; k < K; ++k) {
                const float *c = ks + 5 * k;
                const double dx = __dsub_rn((double)c[0], x0), dy = __dsub_rn((double)c[1], x1),
                             dz = __dsub_rn((double)c[2], x2);
                const double q = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                const double sig = c[3];
                const double den = __dmul_rn(2.0, __dmul_rn(sig, sig));
                const double w = __dmul_rn((double)c[4], attraction_exp(-__ddiv_rn(q, den)));
                d0 = __dadd_rn(d0, __dmul_rn(w, dx));
                d1 = __dadd_rn(d1, __dmul_rn(w, dy));
                d2 = __dadd_rn(d2, __dmul_rn(w, dz));
            }
            const unsigned fx = fixed ? fixed[v] : 0u;
            cand[3 * v] = (fx & 1u) ? pos[3 * v] : __double2float_rn(__dadd_rn(x0, d0));
            cand[3 * v + 1] = (fx & 2u) ? pos[3 * v + 1] : __double2float_rn(__dadd_rn(x1, d1));
            cand[3 * v + 2] = (fx & 4u) ? pos[3 * v + 2] : __double2float_rn(__dadd_rn(x2, d2));
        }
        __syncthreads();
        int folded = 0;
        for (int t = threadIdx.x; t < T && !folded; t += blockDim.x) {
            const int4 tv = P.tets[t];
            folded = orient_d(snap3(cand + 3 * tv.x, P), snap3(cand + 3 * tv.y, P), snap3(cand + 3 * tv.z, P),
                              snap3(cand + 3 * tv.w, P)) <= 0.0;
        }
        if (__syncthreads_or(folded)) break;
        for (int v = threadIdx.x; v < V; v += blockDim.x) {   // each thread keeps its own points
            pos[3 * v] = cand[3 * v];
            pos[3 * v + 1] = cand[3 * v + 1];
            pos[3 * v + 2] = cand[3 * v + 2];
        }
        ++kept;
    }
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
        X[3 * v] = pos[3 * v];
        X[3 * v + 1] = pos[3 * v + 1];
        X[3 * v + 2] = pos[3 * v + 2];
    }
    if (threadIdx.x == 0) rounds_out[2 * sol + mesh] = kept;
}

}  // namespace

size_t init_smem_bytes(int n_points, int n_kernels) { return sizeof(float) * (5 * (size_t)n_kernels + 6 * (size_t)n_points); }

cudaError_t launch_init(const DevProblem *dp, const DevProblem &hp, int n_sol, float *src, float *tgt,
                        const uint8_t *fixed, int n_kernels, const float *kernels, int max_rounds, int *rounds,
                        cudaStream_t st)
{
    const size_t smem = init_smem_bytes(hp.n_points, n_kernels);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_init, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_init<<<2 * n_sol, kInitThreads, smem, st>>>(dp, src, tgt, fixed, n_kernels, kernels, max_rounds, rounds);
    return cudaGetLastError();
}

}  // namespace morea
