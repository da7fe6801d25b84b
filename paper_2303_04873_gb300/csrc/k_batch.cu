// Batched full evaluation of several problems (step a11): one launch of each
// of snap, entries and reduction covers every problem of the batch; the set-up
// and the image/guidance passes already take a problem index per work entry.
// The per-problem results are identical to morea_eval_full's (same per-item
// arithmetic, same reduction order).
#include "morea_device.cuh"

namespace morea {

namespace {

// last problem whose offset (selected by Off) is <= g
template <typename Off>
__device__ __forceinline__ int find_prob(const BatchTable &tb, long long g, Off off)
{
    int lo = 0, hi = tb.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off(tb.p[mid]) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kBlock) k_batch_snap(const DevProblem *__restrict__ probs, const BatchTable tb)
{
    BatchClock *ck = probs[0].clock;
    if (ck && blockIdx.x == 0 && threadIdx.x == 0) {
        // completion clock of this evaluation: start time, item totals, counters cleared
        ck->t0 = global_ns();
        for (int i = 0; i < tb.n; ++i) {
            ck->raster_total[i] = 2 * tb.p[i].n_sol * probs[i].n_tets;
            ck->raster_done[i] = ck->guid_done[i] = ck->guid_total[i] = ck->reduce_done[i] = 0;
            ck->t_raster[i] = ck->t_guid[i] = ck->t_reduce[i] = 0ull;
        }
    }
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < tb.total_verts;
         g += (long long)gridDim.x * blockDim.x) {
        const int pi = find_prob(tb, g, [](const BatchProb &b) { return b.vert_off; });
        const BatchProb &bp = tb.p[pi];
        const DevProblem &P = probs[pi];
        const long long local = g - bp.vert_off;
        const int V = P.n_points;
        const int i = (int)(local / V), v = (int)(local - (long long)i * V);
        int4 *q = const_cast<int4 *>(P.slot_q) + (size_t)i * 2 * V;
        q[v] = snap3(bp.src + 3 * local, P);
        q[V + v] = snap3(bp.tgt + 3 * local, P);
    }
}

__global__ void __launch_bounds__(kBlock) k_batch_entries(const DevProblem *__restrict__ probs, const BatchTable tb,
                                                         WorkEntry *entries)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tb.total_entries;
         e += (long long)gridDim.x * blockDim.x) {
        const int pi = find_prob(tb, e, [](const BatchProb &b) { return b.entry_off; });
        const DevProblem &P = probs[pi];
        const long long local = e - tb.p[pi].entry_off;
        const int V = P.n_points;
        // tet-major within the problem (as k_full_entries): neighbouring
        // items share a region of the images
        const int ns = tb.p[pi].n_sol;
        const int t = (int)(local / ns), i = (int)(local - (long long)t * ns);
        const int4 tv = P.tets[t];
        const int4 *sq = P.slot_q + (size_t)i * 2 * V;
        WorkEntry we;
        we.req = i;
        we.slot = i;
        we.tet = t;
        we.prob = pi;
        const int vid[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            we.q[0][m] = sq[vid[m]];
            we.q[1][m] = sq[V + vid[m]];
        }
        entries[e] = we;
    }
}

template <typename T>
__device__ __forceinline__ T bsum(T v, T *sh)
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

// Per solution of every problem: FP64 sums over its tets in the same order
// as k_reduce_full, the slot's cache and totals, and the objectives.
__global__ void __launch_bounds__(kBlock) k_batch_reduce(const DevProblem *__restrict__ probs, const BatchTable tb,
                                                        const TetOut *__restrict__ tout,
                                                        const RasterOut *__restrict__ rout)
{
    __shared__ double shd[kBlock];
    const int b = blockIdx.x;
    const int pi = find_prob(tb, b, [](const BatchProb &x) { return (long long)x.sol_off; });
    const BatchProb &bp = tb.p[pi];
    const DevProblem &P = probs[pi];
    const int i = b - bp.sol_off;
    const int T = P.n_tets;
    double s_img = 0.0, s_guid = 0.0, s_mag = 0.0;
    long long n_vox = 0, n_gp = 0, n_folded = 0;
    unsigned long long sev = 0;
    morea_tet_record *cache = P.cache + (size_t)i * T;
    for (int t = threadIdx.x; t < T; t += kBlock) {
        const size_t e = (size_t)bp.entry_off + (size_t)t * bp.n_sol + i;
        const TetOut to = tout[e];
        const RasterOut r0 = rout[2 * e], r1 = rout[2 * e + 1];
        morea_tet_record rec;
        rec.e_img[0] = r0.e_img;
        rec.e_img[1] = r1.e_img;
        rec.e_guid[0] = r0.e_guid;
        rec.e_guid[1] = r1.e_guid;
        rec.n_vox[0] = r0.n_vox;
        rec.n_vox[1] = r1.n_vox;
        rec.n_gp[0] = r0.n_gp;
        rec.n_gp[1] = r1.n_gp;
        rec.e_mag = to.e_mag;
        rec.folded = to.folded;
        rec.sev = to.sev;
        cache[t] = rec;
        s_img += (double)rec.e_img[0] + (double)rec.e_img[1];
        s_guid += (double)rec.e_guid[0] + (double)rec.e_guid[1];
        s_mag += (double)rec.e_mag;
        n_vox += (long long)rec.n_vox[0] + rec.n_vox[1];
        n_gp += (long long)rec.n_gp[0] + rec.n_gp[1];
        n_folded += (long long)(((rec.folded & 1u) != 0) + ((rec.folded & 2u) != 0));
        sev += rec.sev;
    }
    s_img = bsum<double>(s_img, shd);
    s_guid = bsum<double>(s_guid, shd);
    s_mag = bsum<double>(s_mag, shd);
    n_vox = bsum<long long>(n_vox, (long long *)shd);
    n_gp = bsum<long long>(n_gp, (long long *)shd);
    n_folded = bsum<long long>(n_folded, (long long *)shd);
    sev = bsum<unsigned long long>(sev, (unsigned long long *)shd);
    if (threadIdx.x == 0) {
        morea_totals mt = {s_img, s_guid, s_mag, n_vox, n_gp, n_folded, sev, 0};
        P.totals[i] = mt;
        double *obj = bp.obj + 3 * i;
        obj[0] = n_vox > 0 ? s_img / (double)n_vox : 0.0;
        obj[1] = s_mag / (10.0 * (double)T);
        double g = 0.0;
        if (P.g_mode == MOREA_G_CONTINUOUS) g = n_vox > 0 ? s_guid / (double)n_vox : 0.0;
        else if (P.g_mode == MOREA_G_PAIR_TRANSFER) g = n_gp > 0 ? s_guid / (double)n_gp : 0.0;
        obj[2] = g;
        bp.folded[i] = n_folded > 0 ? 1 : 0;
        if (bp.severity) {
            const double S = (double)P.S;
            bp.severity[i] = (double)sev / (6.0 * S * S * S);
        }
        BatchClock *ck = P.clock;
        if (ck) {
            __threadfence();                          // this solution's outputs before the stamp
            if (atomicAdd(&ck->reduce_done[pi], 1) + 1 == bp.n_sol) ck->t_reduce[pi] = global_ns();
        }
    }
}

inline int grid_of(long long work)
{
    long long b = (work + kBlock - 1) / kBlock;
    b = std::min<long long>(b, (long long)sm_count() * 16);
    return (int)std::max<long long>(b, 1);
}

}  // namespace

cudaError_t launch_batch_snap(const DevProblem *probs, const BatchTable &tb, cudaStream_t st)
{
    k_batch_snap<<<grid_of(tb.total_verts), kBlock, 0, st>>>(probs, tb);
    return cudaGetLastError();
}

cudaError_t launch_batch_entries(const DevProblem *probs, const BatchTable &tb, WorkEntry *entries, cudaStream_t st)
{
    k_batch_entries<<<grid_of(tb.total_entries), kBlock, 0, st>>>(probs, tb, entries);
    return cudaGetLastError();
}

cudaError_t launch_batch_reduce(const DevProblem *probs, const BatchTable &tb, const TetOut *tout,
                                const RasterOut *rout, cudaStream_t st)
{
    k_batch_reduce<<<tb.total_sols, kBlock, 0, st>>>(probs, tb, tout, rout);
    return cudaGetLastError();
}

}  // namespace morea
