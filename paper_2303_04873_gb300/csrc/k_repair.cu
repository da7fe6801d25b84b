// Repair of folded solutions (Sec. 4.3.1): points of folded tets are moved,
// one at a time, to the best of 64 Gaussian trials when that decreases the
// fold severity of their star.
//
// One warp per solution, because the visits are sequential: a move changes
// which tets are folded when the scan reaches them.  Within a visit the
// lanes share the work: the trial scale (distance to the planes of the faces
// opposite the point) and the current star severity are lane-parallel over
// the star; the 64 trials are two per lane, each evaluated over the whole
// star with exact orientations, and a warp argmax picks the largest
// decrease (lowest trial on ties).  The scan visits the tets 32 at a time
// and re-tests, after every move, which of the remaining tets of the chunk
// are folded.  Scale and trial positions are computed in FP64 with
// explicitly rounded operations, so they equal the plain definition bit for
// bit; orientations are exact.  A coordinate whose axis is fixed for its
// point (on a face of the image box) keeps its value in every trial.
#include "morea_device.cuh"

namespace morea {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kRepairWarps = 4;
constexpr int kTrials = 64;

__device__ __forceinline__ bool tet_folded(const DevProblem &P, const float *X, int t)
{
    const int4 tv = P.tets[t];
    const int4 a = snap3(X + 3 * (size_t)tv.x, P), b = snap3(X + 3 * (size_t)tv.y, P);
    const int4 c = snap3(X + 3 * (size_t)tv.z, P), d = snap3(X + 3 * (size_t)tv.w, P);
    return orient_d(a, b, c, d) <= 0.0;
}

// |orient| if the tet (with v placed at q) is folded, else 0
__device__ __forceinline__ unsigned long long folded_volume(const DevProblem &P, const float *X, int t, int v, int4 q)
{
    const int4 tv = P.tets[t];
    const int4 a = tv.x == v ? q : snap3(X + 3 * (size_t)tv.x, P);
    const int4 b = tv.y == v ? q : snap3(X + 3 * (size_t)tv.y, P);
    const int4 c = tv.z == v ? q : snap3(X + 3 * (size_t)tv.z, P);
    const int4 d = tv.w == v ? q : snap3(X + 3 * (size_t)tv.w, P);
    const double D = orient_d(a, b, c, d);
    return D <= 0.0 ? (unsigned long long)fabs(D) : 0ull;
}

// distance (voxels) from p to the plane of the face of tet t opposite v
__device__ __forceinline__ double opposite_plane_distance(const DevProblem &P, const float *X, int t, int v, int4 p)
{
    const int4 tv = P.tets[t];
    const int ids[4] = {tv.x, tv.y, tv.z, tv.w};
    int4 f[3];
    int n = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (ids[i] != v && n < 3) f[n++] = snap3(X + 3 * (size_t)ids[i], P);
    const long long ux = f[1].x - f[0].x, uy = f[1].y - f[0].y, uz = f[1].z - f[0].z;
    const long long vx = f[2].x - f[0].x, vy = f[2].y - f[0].y, vz = f[2].z - f[0].z;
    const long long nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
    const double nn = __dadd_rn(__dadd_rn(__dmul_rn((double)nx, (double)nx), __dmul_rn((double)ny, (double)ny)),
                                __dmul_rn((double)nz, (double)nz));
    if (nn == 0.0) return INFINITY;
    const long long num = nx * (p.x - f[0].x) + ny * (p.y - f[0].y) + nz * (p.z - f[0].z);
    return __ddiv_rn(__ddiv_rn(fabs((double)num), __dsqrt_rn(nn)), (double)P.S);
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

__global__ void __launch_bounds__(kRepairWarps * 32) k_repair(const DevProblem *__restrict__ dp,
                                                              const int *__restrict__ v2t_off,
                                                              const int *__restrict__ v2t_idx, int n_sol,
                                                              float *src, float *tgt,
                                                              const float *__restrict__ noise, int max_points,
                                                              double scale, const uint8_t *__restrict__ fixed,
                                                              int *moved_out, double *sev_out)
{
    extern __shared__ unsigned done_all[];
    const DevProblem &P = *dp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sol = blockIdx.x * kRepairWarps + warp;
    if (sol >= n_sol) return;                       // warp-uniform
    const int V = P.n_points, T = P.n_tets, W = (V + 31) / 32;
    unsigned *done = done_all + (size_t)warp * W;
    const double floor_s = 1.0 / (double)P.S;
    int moved = 0, visits = 0;
    bool stop = false;
    for (int m = 0; m < 2 && !stop; ++m) {
        float *X = (m == 0 ? src : tgt) + (size_t)sol * V * 3;
        for (int w = lane; w < W; w += 32) done[w] = 0u;
        __syncwarp();
        for (int t0 = 0; t0 < T && !stop; t0 += 32) {
            int cur = -1;                           // last tet of the chunk already handled
            while (!stop) {
                const int t = t0 + lane;
                const bool f = lane > cur && t < T && tet_folded(P, X, t);
                const unsigned mask = __ballot_sync(FULL, f);
                if (!mask) break;
                cur = __ffs(mask) - 1;
                const int4 tv = P.tets[t0 + cur];
                const int vs[4] = {tv.x, tv.y, tv.z, tv.w};
                for (int i = 0; i < 4 && !stop; ++i) {
                    const int v = vs[i];
                    if (done[v >> 5] & (1u << (v & 31))) continue;
                    __syncwarp();
                    if (lane == 0) done[v >> 5] |= 1u << (v & 31);
                    __syncwarp();
                    if (visits >= max_points) {
                        stop = true;
                        break;
                    }
                    const int s0 = v2t_off[v], s1 = v2t_off[v + 1];
                    const int4 p = snap3(X + 3 * (size_t)v, P);
                    // trial scale and the star's severity now (lane-parallel over the star)
                    double dmin = INFINITY;
                    unsigned long long before = 0;
                    for (int s = s0 + lane; s < s1; s += 32) {
                        const int ts = v2t_idx[s];
                        dmin = fmin(dmin, opposite_plane_distance(P, X, ts, v, p));
                        before += folded_volume(P, X, ts, v, p);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) dmin = fmin(dmin, __shfl_xor_sync(FULL, dmin, o));
                    before = warp_sum_u64(before);
                    double sigma = __dmul_rn(scale, dmin);
                    if (!(sigma >= floor_s)) sigma = floor_s;
                    // two trials per lane
                    const float x0 = X[3 * (size_t)v], x1 = X[3 * (size_t)v + 1], x2 = X[3 * (size_t)v + 2];
                    const unsigned fx = fixed ? fixed[v] : 0u;      // axes on a face of the box stay
                    long long best_gain = 0;
                    int best_k = kTrials;
                    float bq[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int k = lane + 32 * h;
                        const float *z = noise + (((size_t)sol * max_points + visits) * kTrials + k) * 3;
                        float q[3];
                        q[0] = (fx & 1u) ? x0 : __double2float_rn(__dadd_rn((double)x0, __dmul_rn(sigma, (double)z[0])));
                        q[1] = (fx & 2u) ? x1 : __double2float_rn(__dadd_rn((double)x1, __dmul_rn(sigma, (double)z[1])));
                        q[2] = (fx & 4u) ? x2 : __double2float_rn(__dadd_rn((double)x2, __dmul_rn(sigma, (double)z[2])));
                        const int4 qs = snap3(q, P);
                        unsigned long long after = 0;
                        for (int s = s0; s < s1; ++s) after += folded_volume(P, X, v2t_idx[s], v, qs);
                        const long long gain = (long long)before - (long long)after;
                        if (gain > best_gain) {         // k grows with h: the lowest k wins ties
                            best_gain = gain;
                            best_k = k;
                            bq[0] = q[0];
                            bq[1] = q[1];
                            bq[2] = q[2];
                        }
                    }
                    // warp argmax: largest gain, then lowest trial index
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const long long g2 = __shfl_xor_sync(FULL, best_gain, o);
                        const int k2 = __shfl_xor_sync(FULL, best_k, o);
                        if (g2 > best_gain || (g2 == best_gain && k2 < best_k)) {
                            best_gain = g2;
                            best_k = k2;
                        }
                    }
                    ++visits;
                    if (best_k >= kTrials) {            // every trial deteriorates: stop
                        stop = true;
                        break;
                    }
                    if (lane == (best_k & 31)) {             // the lane that evaluated the winner
                        X[3 * (size_t)v] = bq[0];
                        X[3 * (size_t)v + 1] = bq[1];
                        X[3 * (size_t)v + 2] = bq[2];
                    }
                    __syncwarp();
                    ++moved;
                }
            }
        }
    }
    // severity of both meshes afterwards
    unsigned long long sev = 0;
    for (int m = 0; m < 2; ++m) {
        const float *X = (m == 0 ? src : tgt) + (size_t)sol * V * 3;
        for (int t = lane; t < T; t += 32) {
            const int4 tv = P.tets[t];
            const double D = orient_d(snap3(X + 3 * (size_t)tv.x, P), snap3(X + 3 * (size_t)tv.y, P),
                                      snap3(X + 3 * (size_t)tv.z, P), snap3(X + 3 * (size_t)tv.w, P));
            if (D <= 0.0) sev += (unsigned long long)fabs(D);
        }
    }
    sev = warp_sum_u64(sev);
    if (lane == 0) {
        const double S = (double)P.S;
        moved_out[sol] = moved;
        sev_out[sol] = (double)sev / (6.0 * S * S * S);
    }
}

}  // namespace

int repair_warps() { return kRepairWarps; }

cudaError_t launch_repair(const DevProblem *dp, const DevProblem &hp, const int *v2t_off, const int *v2t_idx,
                          int n_sol, float *src, float *tgt, const float *noise, int max_points, double scale,
                          const uint8_t *fixed,
                          int *moved, double *severity, cudaStream_t st)
{
    const size_t smem = (size_t)kRepairWarps * ((hp.n_points + 31) / 32) * sizeof(unsigned);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_repair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int blocks = (n_sol + kRepairWarps - 1) / kRepairWarps;
    k_repair<<<blocks, kRepairWarps * 32, smem, st>>>(dp, v2t_off, v2t_idx, n_sol, src, tgt, noise, max_points,
                                                      scale, fixed, moved, severity);
    return cudaGetLastError();
}

}  // namespace morea
