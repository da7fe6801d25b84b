// Estimation and sampling of the FOS elements' distributions per cluster
// (Sec. 3; reading R20), behind morea_sample_elements.
//
// An element (a, b) has 12 variables: source a (x, y, z), source b, target
// a, target b.  Variables on a fixed axis of their point are not modelled
// and keep the parent's value.
//
//   k_estimate  one warp per (cluster, element): lanes 0-11 sum one
//               variable each over the members (member order), lanes own
//               the 78 entries of the maximum-likelihood covariance, and
//               lane 0 factors Sigma + 1e-6 I over the free variables
//               (Cholesky-Banachiewicz, FP64) into the warp's model
//   k_sample    one thread per request: x = mu + c L z rounded to float,
//               written as the two changed points of a partial request
//               (source rows and target rows), so the output feeds
//               morea_eval_partial directly
//
// Member, element and request indices are checked: a model with an index
// out of range is NaN, and so is every request that uses it or that has an
// index out of range itself.
#include <math.h>

#include "morea_internal.cuh"

namespace morea {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kVars = 12;
constexpr int kEstWarps = 8;
constexpr double kRidge = 1e-6;

struct ElemModel {
    double mu[kVars];
    double L[kVars][kVars];              // lower-triangular factor; rows/columns of fixed variables are zero
};

__device__ __forceinline__ void var_of(int l, int a, int b, int &point, int &mesh, int &axis)
{
    point = (l % 6) < 3 ? a : b;
    mesh = l / 6;
    axis = l % 3;
}

__global__ void __launch_bounds__(kEstWarps * 32) k_estimate(int V, int n_pop, const float *__restrict__ src,
                                                             const float *__restrict__ tgt, int C, int csize,
                                                             const int *__restrict__ members, int m,
                                                             const int2 *__restrict__ elements,
                                                             const uint8_t *__restrict__ fixed,
                                                             ElemModel *__restrict__ models)
{
    __shared__ double s_mu[kEstWarps][kVars];
    __shared__ double s_cov[kEstWarps][kVars][kVars];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long pair = (long long)blockIdx.x * kEstWarps + w;
    if (pair >= (long long)C * m) return;                           // warp-uniform
    const int c = (int)(pair / m), e = (int)(pair - (long long)c * m);
    ElemModel &M = models[pair];
    const int2 el = elements[e];
    bool ok = el.x >= 0 && el.x < V && el.y >= 0 && el.y < V;
    const int *mem = members + (size_t)c * csize;
    for (int j = lane; j < csize; j += 32) {
        const int i = mem[j];
        if (i < 0 || i >= n_pop) ok = false;
    }
    ok = __all_sync(FULL, ok);
    if (!ok) {
        for (int q = lane; q < kVars * (kVars + 1); q += 32) (&M.mu[0])[q] = nan("");
        return;
    }
    auto value = [&](int i, int l) -> double {
        int point, mesh, axis;
        var_of(l, el.x, el.y, point, mesh, axis);
        return (double)(mesh == 0 ? src : tgt)[((size_t)i * V + point) * 3 + axis];
    };
    if (lane < kVars) {
        double s = 0.0;
        for (int j = 0; j < csize; ++j) s = __dadd_rn(s, value(mem[j], lane));
        s_mu[w][lane] = __ddiv_rn(s, (double)csize);
    }
    __syncwarp();
    for (int q = lane; q < kVars * (kVars + 1) / 2; q += 32) {
        int r = 0;                                                  // entry q of the lower triangle -> (r, col)
        while ((r + 1) * (r + 2) / 2 <= q) ++r;
        const int col = q - r * (r + 1) / 2;
        double s = 0.0;
        for (int j = 0; j < csize; ++j) {
            const int i = mem[j];
            const double dr = __dsub_rn(value(i, r), s_mu[w][r]);
            const double dc = __dsub_rn(value(i, col), s_mu[w][col]);
            s = __dadd_rn(s, __dmul_rn(dr, dc));
        }
        s_cov[w][r][col] = __ddiv_rn(s, (double)csize);
    }
    __syncwarp();
    if (lane == 0) {
        int idx[kVars], nf = 0;
        const unsigned fa = fixed ? fixed[el.x] : 0u, fb = fixed ? fixed[el.y] : 0u;
        for (int l = 0; l < kVars; ++l) {
            const unsigned f = (l % 6) < 3 ? fa : fb;
            if (!((f >> (l % 3)) & 1u)) idx[nf++] = l;
        }
        for (int r = 0; r < kVars; ++r) {
            M.mu[r] = s_mu[w][r];
            for (int q = 0; q < kVars; ++q) M.L[r][q] = 0.0;
        }
        for (int r = 0; r < nf; ++r) {
            for (int q = 0; q <= r; ++q) {
                const int gr = idx[r], gq = idx[q];
                double s = s_cov[w][gr][gq];
                if (r == q) s = __dadd_rn(s, kRidge);
                for (int t = 0; t < q; ++t) s = __dsub_rn(s, __dmul_rn(M.L[gr][idx[t]], M.L[gq][idx[t]]));
                if (r == q) {
                    M.L[gr][gr] = s > 0.0 ? __dsqrt_rn(s) : 0.0;
                } else {
                    const double d = M.L[gq][gq];
                    M.L[gr][gq] = d > 0.0 ? __ddiv_rn(s, d) : 0.0;
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_sample_elements(int V, int n_pop, const float *__restrict__ src,
                                                         const float *__restrict__ tgt, int C, int m,
                                                         const int2 *__restrict__ elements,
                                                         const uint8_t *__restrict__ fixed,
                                                         const float *__restrict__ cmult, int n_req,
                                                         const int *__restrict__ req_sol,
                                                         const int *__restrict__ req_cluster,
                                                         const int *__restrict__ req_elem,
                                                         const float *__restrict__ z,
                                                         const ElemModel *__restrict__ models, float *new_src,
                                                         float *new_tgt)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_req) return;
    const int sol = req_sol[r], c = req_cluster[r], e = req_elem[r];
    float *os = new_src + (size_t)6 * r, *ot = new_tgt + (size_t)6 * r;   // rows (a, b) of this request
    if (sol < 0 || sol >= n_pop || c < 0 || c >= C || e < 0 || e >= m) {
        for (int q = 0; q < 6; ++q) os[q] = ot[q] = nanf("");
        return;
    }
    const ElemModel &M = models[(size_t)c * m + e];
    const int2 el = elements[e];
    const double cm = cmult[c];
    const float *zr = z + (size_t)kVars * r;
    const unsigned fa = fixed ? fixed[el.x] : 0u, fb = fixed ? fixed[el.y] : 0u;
    for (int l = 0; l < kVars; ++l) {
        int point, mesh, axis;
        var_of(l, el.x, el.y, point, mesh, axis);
        const unsigned f = (l % 6) < 3 ? fa : fb;
        float out;
        if ((f >> axis) & 1u) {
            out = (mesh == 0 ? src : tgt)[((size_t)sol * V + point) * 3 + axis];
        } else {
            double s = 0.0;
            for (int q = 0; q <= l; ++q) s = __dadd_rn(s, __dmul_rn(M.L[l][q], (double)zr[q]));
            out = __double2float_rn(__dadd_rn(M.mu[l], __dmul_rn(cm, s)));
        }
        float *dst = mesh == 0 ? os : ot;
        dst[((l % 6) < 3 ? 0 : 3) + axis] = out;
    }
}

}  // namespace

size_t sample_elements_bytes(int n_clusters, int n_elements)
{
    return sizeof(ElemModel) * (size_t)n_clusters * (size_t)n_elements;
}

cudaError_t launch_sample_elements(int V, int n_pop, const float *src, const float *tgt, int C, int csize,
                                   const int *members, int m, const int *elements, const uint8_t *fixed,
                                   const float *cmult, int n_req, const int *req_sol, const int *req_cluster,
                                   const int *req_elem, const float *z, void *work, float *new_src, float *new_tgt,
                                   cudaStream_t st)
{
    ElemModel *models = static_cast<ElemModel *>(work);
    const long long pairs = (long long)C * m;
    const int2 *el = reinterpret_cast<const int2 *>(elements);
    k_estimate<<<(unsigned)((pairs + kEstWarps - 1) / kEstWarps), kEstWarps * 32, 0, st>>>(
        V, n_pop, src, tgt, C, csize, members, m, el, fixed, models);
    if (n_req > 0)
        k_sample_elements<<<(n_req + 255) / 256, 256, 0, st>>>(V, n_pop, src, tgt, C, m, el, fixed, cmult, n_req,
                                                               req_sol, req_cluster, req_elem, z, models, new_src,
                                                               new_tgt);
    return cudaGetLastError();
}

}  // namespace morea
