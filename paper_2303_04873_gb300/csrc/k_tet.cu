// Tet pass, partial-evaluation scatter/gather and reductions of libmorea.
//
//   k_snap_slots        a0: snap the solutions' points into their slots
//   k_full_entries      a1-a3: per (solution, tet) work entry, fold + magnitude
//                       terms, rasterisation set-up of both copies
//   k_partial_entries   a8: per request, the union of the changed points'
//                       stars (bitmap in shared memory), entries for those tets
//   k_reduce_full       a9: per solution FP64 reduction over tets -> objectives,
//                       cache and totals of the slot
//   k_partial_finalize  a8/a9: per request, totals + sum(new - cached)
//   k_partial_commit    accepted requests: cache, slot coordinates, totals
//   k_check_folds       fold constraint alone
//   k_distance_maps     guidance distance maps (problem set-up)
#include <math.h>

#include "morea_device.cuh"

namespace morea {

namespace {

__global__ void __launch_bounds__(kBlock) k_snap_slots(const DevProblem *__restrict__ dp, int n_sol,
                                                      const int *__restrict__ slot,
                                                      const float *__restrict__ src,
                                                      const float *__restrict__ tgt, int4 *slot_q)
{
    const DevProblem &P = *dp;
    const int V = P.n_points;
    const long long total = (long long)n_sol * V;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(g / V), v = (int)(g - (long long)i * V);
        const int s = slot ? slot[i] : i;
        if (s < 0 || s >= P.max_sol) {
            if (v == 0) atomicOr(P.status, MOREA_DEV_BAD_SLOT);
            continue;
        }
        int4 *q = slot_q + (size_t)s * 2 * V;
        q[v] = snap3(src + 3 * g, P);
        q[V + v] = snap3(tgt + 3 * g, P);
    }
}

// Per-entry work of the tet pass: one thread per (entry, side) builds that
// copy's rasterisation set-up; the side-0 thread also evaluates the fold and
// magnitude terms of the tet.
// With rqueue, the items (entry, side) whose copy is large (item_is_big)
// are also listed for the image pass, which takes them first and the rest
// in their own order, so the pass does not end waiting on a few large
// copies taken late.  The order of the list is arbitrary; an item's result
// does not depend on when it runs.
__global__ void __launch_bounds__(kBlock) k_entry_work(const DevProblem *__restrict__ probs,
                                                      const WorkEntry *__restrict__ entries, RasterSetup *setup,
                                                      TetOut *tout, const int *n_entries_dev, int n_entries_host,
                                                      int *rqueue)
{
    const int n_ent = n_entries_dev ? min(*n_entries_dev, n_entries_host) : n_entries_host;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < 2LL * n_ent;
         g += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(g >> 1), side = (int)(g & 1);
        const WorkEntry &we = entries[e];
        const DevProblem &P = probs[we.prob];
        int4 own[4], oth[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            own[m] = we.q[side][m];
            oth[m] = we.q[1 - side][m];
        }
        RasterSetup su;
        make_setup(own, oth, P, su);
        setup[g] = su;
        if (rqueue && item_is_big(su)) {
            const int pos = atomicAdd(rqueue + kQueueOrderBig, 1);
            rqueue[kQueueList + 2 * (size_t)n_entries_host + pos] = e + side * n_ent;   // raster item index
        }
        if (side == 0) {
            TetOut to;
            tet_terms(own, oth, P, we.tet, to);
            tout[e] = to;
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_full_entries(const DevProblem *__restrict__ dp, int n_sol,
                                                        const int *__restrict__ slot, WorkEntry *entries)
{
    const DevProblem &P = *dp;
    const int T = P.n_tets, V = P.n_points;
    const long long total = (long long)n_sol * T;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        // tet-major: the copies of one tet in all solutions are neighbours in
        // the work list, so the image pass works on one region of the images
        // at a time and they stay in L2 across solutions
        const int t = (int)(e / n_sol), i = (int)(e - (long long)t * n_sol);
        int s = slot ? slot[i] : i;
        const bool bad = s < 0 || s >= P.max_sol;
        if (bad) s = 0;
        const int4 tv = P.tets[t];
        const int4 *sq = P.slot_q + (size_t)s * 2 * V;
        WorkEntry we;
        we.req = i;
        we.slot = s;
        we.tet = t;
        we.prob = 0;
        const int vid[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            we.q[0][m] = sq[vid[m]];
            we.q[1][m] = sq[V + vid[m]];
        }
        entries[e] = we;
    }
}

// deterministic block reduction helpers (fixed tree over kBlock threads)
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *sh)
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

struct Acc {
    double s_img, s_guid, s_mag;
    long long n_vox, n_gp, n_folded;
    unsigned long long sev;
};

__device__ __forceinline__ void acc_add(Acc &a, const morea_tet_record &r, int sign)
{
    a.s_img += sign * ((double)r.e_img[0] + (double)r.e_img[1]);
    a.s_guid += sign * ((double)r.e_guid[0] + (double)r.e_guid[1]);
    a.s_mag += sign * (double)r.e_mag;
    a.n_vox += sign * ((long long)r.n_vox[0] + r.n_vox[1]);
    a.n_gp += sign * ((long long)r.n_gp[0] + r.n_gp[1]);
    a.n_folded += sign * (long long)(((r.folded & 1u) != 0) + ((r.folded & 2u) != 0));
    if (sign > 0) a.sev += r.sev; else a.sev -= r.sev;
}

__device__ __forceinline__ Acc block_acc(Acc a, void *shraw)
{
    Acc o;
    o.s_img = block_sum<double>(a.s_img, (double *)shraw);
    o.s_guid = block_sum<double>(a.s_guid, (double *)shraw);
    o.s_mag = block_sum<double>(a.s_mag, (double *)shraw);
    o.n_vox = block_sum<long long>(a.n_vox, (long long *)shraw);
    o.n_gp = block_sum<long long>(a.n_gp, (long long *)shraw);
    o.n_folded = block_sum<long long>(a.n_folded, (long long *)shraw);
    o.sev = block_sum<unsigned long long>(a.sev, (unsigned long long *)shraw);
    return o;
}

__device__ __forceinline__ morea_tet_record make_record(const TetOut &to, const RasterOut &r0,
                                                        const RasterOut &r1)
{
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
    return rec;
}

// Objectives from totals (Sec. 4.1.1-4.1.3): f_int = sum h / (|P_s| + |P_t|),
// f_mag = sum E / (10 |Delta|), f_guid = sum g / (|P_s| + |P_t|) (continuous)
// or the mean transfer error (pair mode).
__device__ __forceinline__ void objectives(const DevProblem &P, const Acc &a, double *obj, uint8_t *folded,
                                           double *severity)
{
    obj[0] = a.n_vox > 0 ? a.s_img / (double)a.n_vox : 0.0;
    obj[1] = a.s_mag / (10.0 * (double)P.n_tets);
    double g = 0.0;
    if (P.g_mode == MOREA_G_CONTINUOUS) g = a.n_vox > 0 ? a.s_guid / (double)a.n_vox : 0.0;
    else if (P.g_mode == MOREA_G_PAIR_TRANSFER) g = a.n_gp > 0 ? a.s_guid / (double)a.n_gp : 0.0;
    obj[2] = g;
    *folded = a.n_folded > 0 ? 1 : 0;
    if (severity) {
        const double S = (double)P.S;
        *severity = (double)a.sev / (6.0 * S * S * S);
    }
}

__device__ __forceinline__ void bad_outputs(double *obj, uint8_t *folded, double *severity)
{
    obj[0] = obj[1] = obj[2] = nan("");
    *folded = 1;
    if (severity) *severity = nan("");
}

__global__ void __launch_bounds__(kBlock) k_reduce_full(const DevProblem *__restrict__ dp, int n_sol,
                                                       const int *__restrict__ slot,
                                                       const TetOut *__restrict__ tout,
                                                       const RasterOut *__restrict__ rout, double *obj,
                                                       uint8_t *folded, double *severity)
{
    __shared__ double sh[kBlock];
    const DevProblem &P = *dp;
    const int i = blockIdx.x;
    const int T = P.n_tets;
    const int s = slot ? slot[i] : i;
    if (s < 0 || s >= P.max_sol) {
        if (threadIdx.x == 0) bad_outputs(obj + 3 * i, folded + i, severity ? severity + i : nullptr);
        return;
    }
    Acc a = {0.0, 0.0, 0.0, 0, 0, 0, 0};
    morea_tet_record *cache = P.cache + (size_t)s * T;
    for (int t = threadIdx.x; t < T; t += kBlock) {
        const size_t e = (size_t)t * n_sol + i;          // tet-major entries (k_full_entries)
        morea_tet_record rec = make_record(tout[e], rout[2 * e], rout[2 * e + 1]);
        cache[t] = rec;
        acc_add(a, rec, 1);
    }
    Acc tot = block_acc(a, sh);
    if (threadIdx.x == 0) {
        morea_totals mt;
        mt.s_img = tot.s_img;
        mt.s_guid = tot.s_guid;
        mt.s_mag = tot.s_mag;
        mt.n_vox = tot.n_vox;
        mt.n_gp = tot.n_gp;
        mt.n_folded = tot.n_folded;
        mt.sev = tot.sev;
        mt.reserved = 0;
        P.totals[s] = mt;
        objectives(P, tot, obj + 3 * i, folded + i, severity ? severity + i : nullptr);
    }
}

// ---------------------------------------------------------------------------
// partial evaluation
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kBlock) k_partial_entries(
    const DevProblem *__restrict__ dp, int n_req, const int *__restrict__ slot,
    const int *__restrict__ chg_off, const int *__restrict__ chg_pts, const float *__restrict__ chg_src,
    const float *__restrict__ chg_tgt, int max_changed, const int *__restrict__ v2t_off,
    const int *__restrict__ v2t_idx, WorkEntry *entries, int cap, int *counter, ReqInfo *rinfo,
    int *req_chg_pts, int4 *req_chg_q)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_err, s_base, s_m, s_a, s_slot;
    __shared__ int s_scan[kBlock];
    const DevProblem &P = *dp;
    const int r = blockIdx.x, tid = threadIdx.x;
    const int T = P.n_tets, V = P.n_points;
    const int nwords = (T + 31) >> 5;
    int4 *cq = (int4 *)smem;                                  // [max_changed][2]
    int *cid = (int *)(cq + 2 * max_changed);                 // [max_changed]
    unsigned *bits = (unsigned *)(cid + max_changed);         // [nwords]
    if (tid == 0) {
        const int s = slot[r];
        const int a = chg_off[r], b = chg_off[r + 1];
        int err = 0;
        if (s < 0 || s >= P.max_sol) err |= MOREA_DEV_BAD_SLOT;
        if (a < 0 || b < a || b - a > max_changed) err |= MOREA_DEV_TOO_MANY;
        s_err = err;
        s_m = err ? 0 : b - a;
        s_a = a;
        s_slot = s;
    }
    __syncthreads();
    const int m = s_m, a = s_a, s = s_slot;
    for (int c = tid; c < m; c += kBlock) {
        const int v = chg_pts[a + c];
        if (v < 0 || v >= V) atomicOr(&s_err, (int)MOREA_DEV_BAD_POINT);
        cid[c] = v;
        cq[2 * c] = snap3(chg_src + 3 * (size_t)(a + c), P);
        cq[2 * c + 1] = snap3(chg_tgt + 3 * (size_t)(a + c), P);
    }
    for (int w = tid; w < nwords; w += kBlock) bits[w] = 0u;
    __syncthreads();
    for (int c = tid; c < m; c += kBlock)
        for (int d = 0; d < c; ++d)
            if (cid[d] == cid[c]) atomicOr(&s_err, (int)MOREA_DEV_DUPLICATE);
    __syncthreads();
    if (s_err) {
        if (tid == 0) {
            atomicOr(P.status, (unsigned)s_err);
            ReqInfo ri = {0, 0, s_err, s, 0, 0, 0, 0};
            rinfo[r] = ri;
        }
        return;
    }
    // union of the stars of the changed points (dependent tets, Sec. 4.2.1)
    for (int c = tid; c < m; c += kBlock) {
        const int v = cid[c];
        for (int k = v2t_off[v]; k < v2t_off[v + 1]; ++k) {
            const int t = v2t_idx[k];
            atomicOr(&bits[t >> 5], 1u << (t & 31));
        }
    }
    __syncthreads();
    const int chunk = (nwords + kBlock - 1) / kBlock;
    const int w0 = min(nwords, tid * chunk), w1 = min(nwords, w0 + chunk);
    int cnt = 0;
    for (int w = w0; w < w1; ++w) cnt += __popc(bits[w]);
    s_scan[tid] = cnt;
    __syncthreads();
    for (int o = 1; o < kBlock; o <<= 1) {                    // inclusive Hillis-Steele scan
        int v = tid >= o ? s_scan[tid - o] : 0;
        __syncthreads();
        s_scan[tid] += v;
        __syncthreads();
    }
    const int excl = s_scan[tid] - cnt;
    const int total = s_scan[kBlock - 1];
    if (tid == 0) {
        int base = atomicAdd(counter, total);
        if (base + total > cap) {
            s_err = MOREA_DEV_OVERFLOW;
            atomicOr(P.status, MOREA_DEV_OVERFLOW);
        }
        s_base = base;
    }
    __syncthreads();
    if (s_err) {
        if (tid == 0) {
            ReqInfo ri = {0, 0, s_err, s, 0, 0, 0, 0};
            rinfo[r] = ri;
        }
        return;
    }
    // compaction: the owner of each bitmap word writes its tets' ids in order
    int pos = s_base + excl;
    for (int w = w0; w < w1; ++w) {
        unsigned b = bits[w];
        while (b) {
            entries[pos++].tet = (w << 5) + __ffs(b) - 1;
            b &= b - 1;
        }
    }
    __syncthreads();
    // all threads fill the entries: vertices from the request or the slot
    const int4 *sq = P.slot_q + (size_t)s * 2 * V;
    for (int k = tid; k < total; k += kBlock) {
        WorkEntry &we = entries[s_base + k];
        const int t = we.tet;
        const int4 tv = P.tets[t];
        const int vid[4] = {tv.x, tv.y, tv.z, tv.w};
        we.req = r;
        we.slot = s;
        we.prob = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int hit = -1;
            for (int c = 0; c < m; ++c)
                if (cid[c] == vid[q]) { hit = c; break; }
            we.q[0][q] = hit >= 0 ? cq[2 * hit] : sq[vid[q]];
            we.q[1][q] = hit >= 0 ? cq[2 * hit + 1] : sq[V + vid[q]];
        }
    }
    for (int c = tid; c < m; c += kBlock) {
        req_chg_pts[(size_t)r * max_changed + c] = cid[c];
        req_chg_q[2 * ((size_t)r * max_changed + c)] = cq[2 * c];
        req_chg_q[2 * ((size_t)r * max_changed + c) + 1] = cq[2 * c + 1];
    }
    if (tid == 0) {
        ReqInfo ri = {s_base, total, 0, s, m, 0, 0, 0};
        rinfo[r] = ri;
    }
}

__global__ void __launch_bounds__(kBlock) k_partial_finalize(const DevProblem *__restrict__ dp,
                                                            const ReqInfo *__restrict__ rinfo,
                                                            const WorkEntry *__restrict__ entries,
                                                            const TetOut *__restrict__ tout,
                                                            const RasterOut *__restrict__ rout,
                                                            morea_totals *delta, double *obj,
                                                            uint8_t *folded, double *severity)
{
    __shared__ double sh[kBlock];
    const DevProblem &P = *dp;
    const int r = blockIdx.x;
    const ReqInfo ri = rinfo[r];
    if (ri.err) {
        if (threadIdx.x == 0) {
            bad_outputs(obj + 3 * r, folded + r, severity ? severity + r : nullptr);
            morea_totals z = {0.0, 0.0, 0.0, 0, 0, 0, 0, 0};
            delta[r] = z;
        }
        return;
    }
    const int T = P.n_tets;
    const morea_tet_record *cache = P.cache + (size_t)ri.slot * T;
    Acc d = {0.0, 0.0, 0.0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < ri.count; k += kBlock) {
        const size_t e = (size_t)ri.base + k;
        const morea_tet_record nw = make_record(tout[e], rout[2 * e], rout[2 * e + 1]);
        acc_add(d, nw, 1);
        acc_add(d, cache[entries[e].tet], -1);
    }
    Acc dt = block_acc(d, sh);
    if (threadIdx.x == 0) {
        const morea_totals cur = P.totals[ri.slot];
        Acc c;
        c.s_img = cur.s_img + dt.s_img;
        c.s_guid = cur.s_guid + dt.s_guid;
        c.s_mag = cur.s_mag + dt.s_mag;
        c.n_vox = cur.n_vox + dt.n_vox;
        c.n_gp = cur.n_gp + dt.n_gp;
        c.n_folded = cur.n_folded + dt.n_folded;
        c.sev = cur.sev + dt.sev;
        objectives(P, c, obj + 3 * r, folded + r, severity ? severity + r : nullptr);
        morea_totals z = {dt.s_img, dt.s_guid, dt.s_mag, dt.n_vox, dt.n_gp, dt.n_folded, dt.sev, 0};
        delta[r] = z;
    }
}

__global__ void __launch_bounds__(kBlock) k_partial_commit(
    const DevProblem *__restrict__ dp, int n_req, const uint8_t *__restrict__ accept,
    const ReqInfo *__restrict__ rinfo, const WorkEntry *__restrict__ entries, const TetOut *__restrict__ tout,
    const RasterOut *__restrict__ rout, const morea_totals *__restrict__ delta,
    const int *__restrict__ req_chg_pts, const int4 *__restrict__ req_chg_q, int max_changed,
    const int *__restrict__ counter, int cap, int4 *slot_q)
{
    const DevProblem &P = *dp;
    const int T = P.n_tets, V = P.n_points;
    const int n_ent = min(*counter, cap);
    const long long span = max((long long)n_ent, (long long)n_req * max_changed);
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < span;
         g += (long long)gridDim.x * blockDim.x) {
        if (g < n_ent) {
            const WorkEntry &we = entries[g];
            if (we.req < 0 || we.req >= n_req) continue;
            const ReqInfo ri = rinfo[we.req];
            if (!ri.err && accept[we.req])
                P.cache[(size_t)we.slot * T + we.tet] = make_record(tout[g], rout[2 * g], rout[2 * g + 1]);
        }
        if (g < (long long)n_req * max_changed) {
            const int r = (int)(g / max_changed), c = (int)(g - (long long)r * max_changed);
            const ReqInfo ri = rinfo[r];
            if (!ri.err && accept[r] && c < ri.nchg) {
                const int v = req_chg_pts[g];
                int4 *q = slot_q + (size_t)ri.slot * 2 * V;
                q[v] = req_chg_q[2 * g];
                q[V + v] = req_chg_q[2 * g + 1];
            }
        }
        if (g < n_req) {
            const ReqInfo ri = rinfo[g];
            if (!ri.err && accept[g]) {
                const morea_totals d = delta[g];
                morea_totals *t = P.totals + ri.slot;
                atomicAdd(&t->s_img, d.s_img);
                atomicAdd(&t->s_guid, d.s_guid);
                atomicAdd(&t->s_mag, d.s_mag);
                atomicAdd((unsigned long long *)&t->n_vox, (unsigned long long)d.n_vox);
                atomicAdd((unsigned long long *)&t->n_gp, (unsigned long long)d.n_gp);
                atomicAdd((unsigned long long *)&t->n_folded, (unsigned long long)d.n_folded);
                atomicAdd((unsigned long long *)&t->sev, (unsigned long long)d.sev);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// fold constraint alone, read-back, distance maps
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kBlock) k_check_folds(const DevProblem *__restrict__ dp,
                                                       const float *__restrict__ src,
                                                       const float *__restrict__ tgt, uint8_t *folded,
                                                       double *severity)
{
    __shared__ unsigned long long sh[kBlock];
    const DevProblem &P = *dp;
    const int i = blockIdx.x, V = P.n_points, T = P.n_tets;
    const float *ps = src + (size_t)i * V * 3, *pt = tgt + (size_t)i * V * 3;
    unsigned long long nf = 0, sev = 0;
    for (int t = threadIdx.x; t < T; t += kBlock) {
        const int4 tv = P.tets[t];
        const int vid[4] = {tv.x, tv.y, tv.z, tv.w};
        int4 qs[4], qt[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            qs[m] = snap3(ps + 3 * vid[m], P);
            qt[m] = snap3(pt + 3 * vid[m], P);
        }
        const double Ds = orient_d(qs[0], qs[1], qs[2], qs[3]);
        const double Dt = orient_d(qt[0], qt[1], qt[2], qt[3]);
        if (Ds <= 0.0) { ++nf; sev += (unsigned long long)(-Ds); }
        if (Dt <= 0.0) { ++nf; sev += (unsigned long long)(-Dt); }
    }
    nf = block_sum<unsigned long long>(nf, sh);
    sev = block_sum<unsigned long long>(sev, sh);
    if (threadIdx.x == 0) {
        folded[i] = nf > 0 ? 1 : 0;
        if (severity) {
            const double S = (double)P.S;
            severity[i] = (double)sev / (6.0 * S * S * S);
        }
    }
}

__global__ void k_gather_records(const morea_tet_record *__restrict__ cache, int T, int max_sol, int n_sol,
                                 const int *__restrict__ slot, morea_tet_record *out)
{
    const long long total = (long long)n_sol * T;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(g / T), t = (int)(g - (long long)i * T);
        const int s = slot ? slot[i] : i;
        if (s >= 0 && s < max_sol) out[g] = cache[(size_t)s * T + t];
    }
}

__global__ void k_gather_totals(const morea_totals *__restrict__ tot, int max_sol, int n_sol,
                                const int *__restrict__ slot, morea_totals *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_sol) return;
    const int s = slot ? slot[i] : i;
    if (s >= 0 && s < max_sol) out[i] = tot[s];
}

// Objectives of committed slots from their running totals (a9).
__global__ void k_slot_objectives(const DevProblem *__restrict__ dp, int n_sol, const int *__restrict__ slot,
                                  double *obj, uint8_t *folded, double *severity)
{
    const DevProblem &P = *dp;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_sol) return;
    const int s = slot ? slot[i] : i;
    if (s < 0 || s >= P.max_sol) {
        bad_outputs(obj + 3 * i, folded + i, severity ? severity + i : nullptr);
        return;
    }
    const morea_totals t = P.totals[s];
    const Acc a = {t.s_img, t.s_guid, t.s_mag, t.n_vox, t.n_gp, t.n_folded, t.sev};
    objectives(P, a, obj + 3 * i, folded + i, severity ? severity + i : nullptr);
}

// Distance map of each contour group (Sec. 4.1.3 / App. A.3): Euclidean
// distance from each voxel centre to the nearest point of the group, and the
// per-voxel mask of groups whose truncation band (distance < r) holds it.
__global__ void __launch_bounds__(kBlock) k_distance_maps(int nx, int ny, int nz, int G, float r,
                                                         const float4 *__restrict__ pts,
                                                         const int *__restrict__ goff, float *dmap,
                                                         uint8_t *band)
{
    const long long N = (long long)nx * ny * nz;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % nx);
        const int j = (int)((idx / nx) % ny);
        const int k = (int)(idx / ((long long)nx * ny));
        unsigned mask = 0;
        for (int g = 0; g < G; ++g) {
            float best = INFINITY;
            for (int p = goff[g]; p < goff[g + 1]; ++p) {
                const float4 q = pts[p];
                const float dx = (float)i - q.x, dy = (float)j - q.y, dz = (float)k - q.z;
                best = fminf(best, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
            }
            const float d = sqrtf(best);
            dmap[(size_t)g * N + idx] = d;
            if (d < r) mask |= 1u << g;
        }
        band[idx] = (uint8_t)mask;
    }
}

__global__ void __launch_bounds__(kBlock) k_count_visits(const RasterOut *__restrict__ rout,
                                                        const int *n_entries_dev, int n_entries_host,
                                                        unsigned long long *visits)
{
    __shared__ unsigned long long sh[kBlock];
    const int n_ent = n_entries_dev ? min(*n_entries_dev, n_entries_host) : n_entries_host;
    unsigned long long c = 0;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < 2LL * n_ent;
         g += (long long)gridDim.x * blockDim.x)
        c += (unsigned long long)rout[g].n_vox;
    c = block_sum<unsigned long long>(c, sh);
    if (threadIdx.x == 0 && c) atomicAdd(visits, c);
}

// Quad copy (quad_cells layout): one element per padded cell, the four
// values of its z-plane with every index clamped into the image, so one
// 16-byte (FP32) or 8-byte (FP16) load brings one plane of the 2x2x2
// neighbourhood of any position in [-1, n) per axis.
template <typename TI, typename QT>
__device__ __forceinline__ QT quad_of(const TI *img, int i00, int i10, int i01, int i11);

template <>
__device__ __forceinline__ float4 quad_of<float, float4>(const float *img, int i00, int i10, int i01, int i11)
{
    return make_float4(img[i00], img[i10], img[i01], img[i11]);
}

template <>
__device__ __forceinline__ uint2 quad_of<unsigned short, uint2>(const unsigned short *img, int i00, int i10, int i01,
                                                              int i11)
{
    return make_uint2((unsigned)img[i00] | ((unsigned)img[i10] << 16), (unsigned)img[i01] | ((unsigned)img[i11] << 16));
}

template <typename TI, typename QT>
__global__ void __launch_bounds__(kBlock) k_build_quads(const TI *__restrict__ img, int nx, int ny, int nz, QT *quad)
{
    const long long cells = (long long)(nx + 1) * (ny + 1) * (nz + 2);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < cells;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % (nx + 1)) - 1, y = (int)((idx / (nx + 1)) % (ny + 1)) - 1;
        const int z = (int)(idx / ((long long)(nx + 1) * (ny + 1))) - 1;
        const int x0 = min(max(x, 0), nx - 1), x1 = min(x + 1, nx - 1);
        const int y0 = min(max(y, 0), ny - 1), y1 = min(y + 1, ny - 1);
        const int zo = min(max(z, 0), nz - 1) * ny;
        quad[idx] = quad_of<TI, QT>(img, (zo + y0) * nx + x0, (zo + y0) * nx + x1, (zo + y1) * nx + x0,
                                    (zo + y1) * nx + x1);
    }
}

// x-range of the voxels of each image row that lie in some guidance band.
__global__ void __launch_bounds__(kBlock) k_band_rows(const uint8_t *__restrict__ band, int nx, int ny, int nz,
                                                     short2 *bandrow)
{
    const int rows = ny * nz;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < rows; row += gridDim.x * blockDim.x) {
        const uint8_t *b = band + (size_t)row * nx;
        int lo = 32767, hi = -1;
        for (int x = 0; x < nx; ++x)
            if (b[x]) {
                lo = min(lo, x);
                hi = x;
            }
        bandrow[row] = make_short2((short)lo, (short)hi);
    }
}

// Distance word of each band record: the voxel's own distance to the lowest
// guidance group whose band holds it (the first term of its guidance sum).
__global__ void __launch_bounds__(kBlock) k_band_records(const float *__restrict__ dmap, const int *__restrict__ start,
                                                        int nx, int rows, size_t n_vox, int2 *rec)
{
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < rows; row += gridDim.x * blockDim.x) {
        const int a = start[row], b = start[row + 1];
        for (int i = a; i < b; ++i) {
            const int2 r = rec[i];
            const int x = r.x & 0xffff, g = __ffs(r.x >> 16) - 1;
            rec[i].y = __float_as_int(dmap[(size_t)g * n_vox + (size_t)row * nx + x]);
        }
    }
}

// Surrogate input of each partial candidate: per vertex the displacement
// target - source (voxel units, snapped coordinates) of the slot's committed
// solution with the request's moved points replaced.
__global__ void __launch_bounds__(kBlock) k_partial_features(const DevProblem *__restrict__ dp,
                                                            const int *__restrict__ slot,
                                                            const int *__restrict__ chg_off,
                                                            const int *__restrict__ chg_pts,
                                                            const float *__restrict__ chg_src,
                                                            const float *__restrict__ chg_tgt, float *out)
{
    const DevProblem &P = *dp;
    const int r = blockIdx.x, V = P.n_points;
    const int s = slot[r];
    float *o = out + (size_t)r * V * 3;
    const float inv_s = 1.0f / (float)P.S;
    if (s < 0 || s >= P.max_sol) {
        for (int v = threadIdx.x; v < 3 * V; v += kBlock) o[v] = __int_as_float(0x7fc00000);
        if (threadIdx.x == 0) atomicOr(P.status, MOREA_DEV_BAD_SLOT);
        return;
    }
    const int4 *sq = P.slot_q + (size_t)s * 2 * V;
    for (int v = threadIdx.x; v < V; v += kBlock) {
        const int4 a = sq[v], b = sq[V + v];
        o[3 * v] = (float)(b.x - a.x) * inv_s;
        o[3 * v + 1] = (float)(b.y - a.y) * inv_s;
        o[3 * v + 2] = (float)(b.z - a.z) * inv_s;
    }
    __syncthreads();
    const int a0 = chg_off[r], a1 = chg_off[r + 1];
    for (int c = a0 + threadIdx.x; c < a1; c += kBlock) {
        const int v = chg_pts[c];
        if (v < 0 || v >= V) {
            atomicOr(P.status, MOREA_DEV_BAD_POINT);
            continue;
        }
        const int4 a = snap3(chg_src + 3 * (size_t)c, P), b = snap3(chg_tgt + 3 * (size_t)c, P);
        o[3 * v] = (float)(b.x - a.x) * inv_s;
        o[3 * v + 1] = (float)(b.y - a.y) * inv_s;
        o[3 * v + 2] = (float)(b.z - a.z) * inv_s;
    }
}

inline int grid_for(long long work, int block = kBlock)
{
    long long b = (work + block - 1) / block;
    long long cap = (long long)sm_count() * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

cudaError_t launch_snap_slots(const DevProblem *dp, const DevProblem &hp, int n_sol, const int *slot,
                              const float *src, const float *tgt, int4 *slot_q, int, cudaStream_t st)
{
    k_snap_slots<<<grid_for((long long)n_sol * hp.n_points), kBlock, 0, st>>>(dp, n_sol, slot, src, tgt,
                                                                             slot_q);
    return cudaGetLastError();
}

cudaError_t launch_full_entries(const DevProblem *dp, const DevProblem &hp, int n_sol, const int *slot,
                                WorkEntry *entries, RasterSetup *setup, TetOut *tout, cudaStream_t st)
{
    k_full_entries<<<grid_for((long long)n_sol * hp.n_tets), kBlock, 0, st>>>(dp, n_sol, slot, entries);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_entry_work(dp, entries, setup, tout, nullptr, n_sol * hp.n_tets, nullptr, st);
}

cudaError_t launch_entry_work(const DevProblem *dp, const WorkEntry *entries, RasterSetup *setup, TetOut *tout,
                              const int *n_entries_dev, int n_entries_host, int *rqueue, cudaStream_t st)
{
    k_entry_work<<<grid_for(2LL * n_entries_host), kBlock, 0, st>>>(dp, entries, setup, tout, n_entries_dev,
                                                                    n_entries_host, rqueue);
    return cudaGetLastError();
}

cudaError_t launch_build_quads(const DevProblem &hp, int side, void *quad, cudaStream_t st)
{
    const long long cells = quad_cells(hp.nx, hp.ny, hp.nz);
    if (hp.dtype == MOREA_F16)
        k_build_quads<unsigned short, uint2><<<grid_for(cells), kBlock, 0, st>>>(
            (const unsigned short *)hp.img[side], hp.nx, hp.ny, hp.nz, (uint2 *)quad);
    else
        k_build_quads<float, float4><<<grid_for(cells), kBlock, 0, st>>>((const float *)hp.img[side], hp.nx, hp.ny,
                                                                       hp.nz, (float4 *)quad);
    return cudaGetLastError();
}

cudaError_t launch_band_rows(const DevProblem &hp, int side, short2 *bandrow, cudaStream_t st)
{
    k_band_rows<<<grid_for((long long)hp.ny * hp.nz), kBlock, 0, st>>>(hp.band[side], hp.nx, hp.ny, hp.nz, bandrow);
    return cudaGetLastError();
}

cudaError_t launch_band_records(const DevProblem &hp, int side, int2 *rec, cudaStream_t st)
{
    const int rows = hp.ny * hp.nz;
    k_band_records<<<grid_for(rows), kBlock, 0, st>>>(hp.dmap[side], hp.band_start[side], hp.nx, rows,
                                                      (size_t)hp.nx * hp.ny * hp.nz, rec);
    return cudaGetLastError();
}

cudaError_t launch_reduce_full(const DevProblem *dp, const DevProblem &, int n_sol, const int *slot,
                               const TetOut *tout, const RasterOut *rout, double *obj, uint8_t *folded,
                               double *severity, cudaStream_t st)
{
    k_reduce_full<<<n_sol, kBlock, 0, st>>>(dp, n_sol, slot, tout, rout, obj, folded, severity);
    return cudaGetLastError();
}

size_t partial_smem_bytes(int n_tets, int max_changed)
{
    return (size_t)max_changed * (2 * sizeof(int4) + sizeof(int)) + sizeof(unsigned) * ((n_tets + 31) / 32);
}

cudaError_t launch_partial_entries(const DevProblem *dp, const DevProblem &hp, int n_req, const int *slot,
                                   const int *chg_off, const int *chg_pts, const float *chg_src,
                                   const float *chg_tgt, int, int max_changed, const int *v2t_off,
                                   const int *v2t_idx, WorkEntry *entries, RasterSetup *setup,
                                   TetOut *tout, int cap_entries, int *counter, ReqInfo *rinfo,
                                   int *req_chg_pts, int4 *req_chg_q, int *rqueue, cudaStream_t st)
{
    const size_t smem = partial_smem_bytes(hp.n_tets, max_changed);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_partial_entries, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_partial_entries<<<n_req, kBlock, smem, st>>>(dp, n_req, slot, chg_off, chg_pts, chg_src, chg_tgt,
                                                   max_changed, v2t_off, v2t_idx, entries, cap_entries, counter,
                                                   rinfo, req_chg_pts, req_chg_q);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_entry_work(dp, entries, setup, tout, counter, cap_entries, rqueue, st);
}

cudaError_t launch_partial_finalize(const DevProblem *dp, const DevProblem &, int n_req, const ReqInfo *rinfo,
                                    const WorkEntry *entries, const TetOut *tout, const RasterOut *rout,
                                    morea_totals *delta, double *obj, uint8_t *folded, double *severity,
                                    cudaStream_t st)
{
    k_partial_finalize<<<n_req, kBlock, 0, st>>>(dp, rinfo, entries, tout, rout, delta, obj, folded,
                                                 severity);
    return cudaGetLastError();
}

cudaError_t launch_partial_commit(const DevProblem *dp, const DevProblem &, int n_req, const uint8_t *accept,
                                  const ReqInfo *rinfo, const WorkEntry *entries, const TetOut *tout,
                                  const RasterOut *rout, const morea_totals *delta, const int *req_chg_pts,
                                  const int4 *req_chg_q, int max_changed, const int *counter, int cap,
                                  int4 *slot_q, cudaStream_t st)
{
    k_partial_commit<<<sm_count() * 4, kBlock, 0, st>>>(dp, n_req, accept, rinfo, entries, tout, rout, delta,
                                                        req_chg_pts, req_chg_q, max_changed, counter, cap,
                                                        slot_q);
    return cudaGetLastError();
}

cudaError_t launch_check_folds(const DevProblem *dp, const DevProblem &, int n_sol, const float *src,
                               const float *tgt, uint8_t *folded, double *severity, cudaStream_t st)
{
    k_check_folds<<<n_sol, kBlock, 0, st>>>(dp, src, tgt, folded, severity);
    return cudaGetLastError();
}

cudaError_t launch_gather_records(const DevProblem &hp, int n_sol, const int *slot, morea_tet_record *out,
                                  cudaStream_t st)
{
    k_gather_records<<<grid_for((long long)n_sol * hp.n_tets), kBlock, 0, st>>>(hp.cache, hp.n_tets,
                                                                               hp.max_sol, n_sol, slot, out);
    return cudaGetLastError();
}

cudaError_t launch_gather_totals(const DevProblem &hp, int n_sol, const int *slot, morea_totals *out,
                                 cudaStream_t st)
{
    k_gather_totals<<<(n_sol + kBlock - 1) / kBlock, kBlock, 0, st>>>(hp.totals, hp.max_sol, n_sol, slot, out);
    return cudaGetLastError();
}

cudaError_t launch_slot_objectives(const DevProblem *dp, int n_sol, const int *slot, double *obj, uint8_t *folded,
                                  double *severity, cudaStream_t st)
{
    k_slot_objectives<<<(n_sol + kBlock - 1) / kBlock, kBlock, 0, st>>>(dp, n_sol, slot, obj, folded, severity);
    return cudaGetLastError();
}

cudaError_t launch_count_visits(const RasterOut *rout, const int *n_entries_dev, int n_entries_host,
                                unsigned long long *visits, cudaStream_t st)
{
    k_count_visits<<<sm_count() * 2, kBlock, 0, st>>>(rout, n_entries_dev, n_entries_host, visits);
    return cudaGetLastError();
}

cudaError_t launch_partial_features(const DevProblem *dp, int n_req, const int *slot, const int *chg_off,
                                    const int *chg_pts, const float *chg_src, const float *chg_tgt, float *out,
                                    cudaStream_t st)
{
    k_partial_features<<<n_req, kBlock, 0, st>>>(dp, slot, chg_off, chg_pts, chg_src, chg_tgt, out);
    return cudaGetLastError();
}

cudaError_t launch_distance_maps(const DevProblem &hp, const float4 *pts, const int *goff, float *dmap,
                                 uint8_t *band, cudaStream_t st)
{
    const long long N = (long long)hp.nx * hp.ny * hp.nz;
    k_distance_maps<<<grid_for(N), kBlock, 0, st>>>(hp.nx, hp.ny, hp.nz, hp.G, hp.r, pts, goff, dmap, band);
    return cudaGetLastError();
}

}  // namespace morea
