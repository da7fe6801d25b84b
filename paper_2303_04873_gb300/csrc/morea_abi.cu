// Host side of the libmorea C ABI (include/morea.h): problem validation and
// set-up, device allocation, and the launch sequence of each entry point.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "morea_host.h"

using namespace morea;

namespace {

// Same snapping rule as the kernels: clamp to [-0.5, n-0.5], then
// rint(x 2^k) + 2^(k-1), round half to even.
int host_snap1(float x, int n, int kbits)
{
    float c = std::fmin(std::fmax(x, -0.5f), (float)n - 0.5f);
    return (int)std::nearbyint(c * (float)(1 << kbits)) + (1 << (kbits - 1));
}

long long host_orient(const int *a, const int *b, const int *c, const int *d)
{
    long long bx = b[0] - a[0], by = b[1] - a[1], bz = b[2] - a[2];
    long long cx = c[0] - a[0], cy = c[1] - a[1], cz = c[2] - a[2];
    long long dx = d[0] - a[0], dy = d[1] - a[1], dz = d[2] - a[2];
    return bx * (cy * dz - cz * dy) + by * (cz * dx - cx * dz) + bz * (cx * dy - cy * dx);
}

// Severity is accumulated exactly in 64 bits: require 4 T N 8^k < 2^63.
bool severity_fits(long long T, long long N, int k)
{
    return std::log2(4.0) + std::log2((double)T) + std::log2((double)N) + 3.0 * k < 63.0;
}

}  // namespace

// Snapping grid 2^-k of a problem (reading R1): a requested k must keep
// max(n) 2^k <= 65536 and the exact severity sum in 64 bits; 0 asks for the
// largest k <= 8 that does.  Returns -1 when no k qualifies.
int morea::choose_subvoxel_bits(int requested, int nx, int ny, int nz, long long n_tets)
{
    const long long nmax = std::max(nx, std::max(ny, nz));
    const long long N = (long long)nx * ny * nz;
    int k = requested;
    if (k == 0) {
        k = 8;
        while (k > 2 && ((nmax << k) > 65536 || !severity_fits(n_tets, N, k))) --k;
    }
    if (k < 2 || k > 14 || (nmax << k) > 65536 || !severity_fits(n_tets, N, k)) return -1;
    return k;
}

namespace {

morea_status from_cuda(cudaError_t e) { return e == cudaSuccess ? MOREA_OK : MOREA_ECUDA; }

// Rasterisation launch wrapped by the optional instrumentation.
cudaError_t timed_raster(morea_problem *p, const int *n_dev, int n_host, int grid, bool ordered, cudaStream_t st)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (p->prof & 1u) {
        while (p->ev.size() < p->ev_used + 2) {
            cudaEvent_t e = nullptr;
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return r;
            p->ev.push_back(e);
        }
        a = p->ev[p->ev_used];
        b = p->ev[p->ev_used + 1];
        p->ev_used += 2;
        cudaError_t r = cudaEventRecord(a, st);
        if (r != cudaSuccess) return r;
    }
    cudaError_t e = launch_raster(p->dp, p->hp, p->entries, p->setup, p->rout, p->bandrows, n_dev, n_host, grid,
                                  p->launch.chunk, p->queue, ordered, nullptr, st);
    if (e == cudaSuccess && (p->prof & 1u)) e = cudaEventRecord(b, st);
    if (e == cudaSuccess && (p->prof & 2u)) e = launch_count_visits(p->rout, n_dev, n_host, p->visits, st);
    return e;
}

}  // namespace

extern "C" {

const char *morea_status_string(morea_status s)
{
    switch (s) {
    case MOREA_OK: return "ok";
    case MOREA_EINVAL: return "invalid argument";
    case MOREA_ENOMEM: return "out of memory";
    case MOREA_ECUDA: return "CUDA runtime error";
    case MOREA_ETIMEOUT: return "bounded device wait gave up";
    case MOREA_ENOTIMPL: return "not implemented";
    case MOREA_EDEVICE: return "device status word reported invalid input";
    }
    return "unknown status";
}

morea_status morea_destroy_problem(morea_problem *p)
{
    if (!p) return MOREA_OK;
    DeviceGuard g(p->device);
    cudaError_t first = cudaSuccess;
    for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
    for (void *m : p->allocs) {
        cudaError_t e = cudaFree(m);
        if (first == cudaSuccess) first = e;
    }
    delete p;
    return from_cuda(first);
}

morea_status morea_create_problem(const morea_problem_desc *d, void *stream, morea_problem **out)
{
    if (!out) return MOREA_EINVAL;
    *out = nullptr;
    if (!d) return MOREA_EINVAL;
    // ---- validation (nothing is allocated before this passes) ----
    if (d->nx < 2 || d->ny < 2 || d->nz < 2) return MOREA_EINVAL;
    if (d->dtype != MOREA_F32 && d->dtype != MOREA_F16) return MOREA_EINVAL;
    if (!d->image_s || !d->image_t) return MOREA_EINVAL;
    if (d->n_points < 4 || d->n_tets < 1 || !d->tets || !d->ref_points) return MOREA_EINVAL;
    if (d->h_mode != MOREA_H_PLAIN_SSD && d->h_mode != MOREA_H_MOREA_FG) return MOREA_EINVAL;
    if (d->g_mode < MOREA_G_CONTINUOUS || d->g_mode > MOREA_G_OFF) return MOREA_EINVAL;
    if (d->estimator != MOREA_EST_VOXELS && d->estimator != MOREA_EST_SAMPLED) return MOREA_EINVAL;
    if (d->estimator == MOREA_EST_SAMPLED &&
        (d->h_mode != MOREA_H_PLAIN_SSD || d->g_mode == MOREA_G_PAIR_TRANSFER || std::isnan(d->sampling_rate) ||
         d->sampling_rate > 1.0e6f))
        return MOREA_EINVAL;
    if (d->n_guid < 0 || (d->n_guid > 0 && (!d->guid_s || !d->guid_t))) return MOREA_EINVAL;
    if (std::isnan(d->trunc_radius)) return MOREA_EINVAL;
    if (d->max_solutions < 1 || d->max_requests < 0 || d->max_changed < 0 || d->max_changed > 1024)
        return MOREA_EINVAL;
    if (d->tissue_factor && d->n_labels < 1) return MOREA_EINVAL;
    if (d->tissue_mask && (!d->tissue_factor || d->n_labels > kMaxTissueLabels)) return MOREA_EINVAL;
    const int nx = d->nx, ny = d->ny, nz = d->nz;
    const long long N = (long long)nx * ny * nz;
    const int V = d->n_points, T = d->n_tets;
    const int k = choose_subvoxel_bits(d->subvoxel_bits, nx, ny, nz, T);
    if (k < 0) return MOREA_EINVAL;
    if (d->tissue_mask)
        for (long long v = 0; v < N; ++v)
            if (d->tissue_mask[v] >= d->n_labels) return MOREA_EINVAL;
    int G = 0;
    for (int m = 0; m < d->n_guid; ++m) {
        const int g = d->guid_group ? d->guid_group[m] : 0;
        if (g < 0 || g >= kMaxGroups) return MOREA_EINVAL;
        G = std::max(G, g + 1);
    }
    if (N * std::max(G, 1) >= (1LL << 31)) return MOREA_EINVAL;
    const int max_sol = d->max_solutions;
    const int max_req = d->max_requests > 0 ? d->max_requests : max_sol;
    const int max_changed = d->max_changed > 0 ? d->max_changed : 64;
    if (partial_smem_bytes(T, max_changed) > 200 * 1024) return MOREA_EINVAL;

    // topology: positive reference orientation, labels, vertex -> tet stars
    std::vector<int4> tets(T);
    std::vector<float> cdelta(T);
    std::vector<int> qref((size_t)V * 3);
    for (int v = 0; v < V; ++v) {
        qref[3 * v] = host_snap1(d->ref_points[3 * v], nx, k);
        qref[3 * v + 1] = host_snap1(d->ref_points[3 * v + 1], ny, k);
        qref[3 * v + 2] = host_snap1(d->ref_points[3 * v + 2], nz, k);
    }
    std::vector<int> star_cnt(V + 1, 0);
    for (int t = 0; t < T; ++t) {
        int v[4];
        for (int m = 0; m < 4; ++m) {
            v[m] = d->tets[4 * t + m];
            if (v[m] < 0 || v[m] >= V) return MOREA_EINVAL;
        }
        const long long D = host_orient(&qref[3 * v[0]], &qref[3 * v[1]], &qref[3 * v[2]], &qref[3 * v[3]]);
        if (D == 0) return MOREA_EINVAL;
        if (D < 0) std::swap(v[2], v[3]);
        tets[t] = make_int4(v[0], v[1], v[2], v[3]);
        const int lab = d->tet_label ? d->tet_label[t] : 0;
        if (d->tissue_factor) {
            if (lab < 0 || lab >= d->n_labels) return MOREA_EINVAL;
            cdelta[t] = (float)d->tissue_factor[lab];
        } else {
            cdelta[t] = 1.0f;
        }
        for (int m = 0; m < 4; ++m) star_cnt[v[m] + 1] += 1;
    }
    std::vector<int> v2t_off(V + 1, 0);
    int max_star = 0;
    for (int v = 0; v < V; ++v) {
        v2t_off[v + 1] = v2t_off[v] + star_cnt[v + 1];
        max_star = std::max(max_star, star_cnt[v + 1]);
    }
    std::vector<int> v2t_idx(v2t_off[V]);
    {
        std::vector<int> fill(v2t_off.begin(), v2t_off.end() - 1);
        for (int t = 0; t < T; ++t) {
            const int vv[4] = {tets[t].x, tets[t].y, tets[t].z, tets[t].w};
            for (int m = 0; m < 4; ++m) v2t_idx[fill[vv[m]]++] = t;
        }
    }
    const long long per_req = std::min<long long>(T, (long long)max_changed * std::max(max_star, 1));
    const long long cap = std::max<long long>((long long)max_sol * T, (long long)max_req * per_req);
    if (cap > (1LL << 30)) return MOREA_EINVAL;

    // guidance: weights, snapped points, buckets, group-sorted points
    const double r = d->trunc_radius > 0.0 ? d->trunc_radius : 0.025 * (double)nx;
    float wgt[kMaxGroups] = {0};
    std::vector<int> gcount(std::max(G, 1), 0);
    for (int m = 0; m < d->n_guid; ++m) gcount[d->guid_group ? d->guid_group[m] : 0] += 1;
    for (int g = 0; g < G; ++g) wgt[g] = (float)((double)gcount[g] / (double)d->n_guid);
    const int S = 1 << k, H = 1 << (k - 1), cshift = k + 3;
    const int cgx = ((nx * S) >> cshift) + 1, cgy = ((ny * S) >> cshift) + 1, cgz = ((nz * S) >> cshift) + 1;
    const int n_cells = cgx * cgy * cgz;
    std::vector<int4> gq[2];
    std::vector<float4> gp[2];
    std::vector<int> cell_start[2], cell_pts[2];
    for (int side = 0; side < 2; ++side) {
        const float *src = side == 0 ? d->guid_s : d->guid_t;
        gq[side].resize(std::max(d->n_guid, 1));
        gp[side].resize(std::max(d->n_guid, 1));
        cell_start[side].assign(n_cells + 1, 0);
        cell_pts[side].resize(std::max(d->n_guid, 1));
        std::vector<int> cell_of(std::max(d->n_guid, 1));
        for (int m = 0; m < d->n_guid; ++m) {
            const int qx = host_snap1(src[3 * m], nx, k), qy = host_snap1(src[3 * m + 1], ny, k),
                      qz = host_snap1(src[3 * m + 2], nz, k);
            gq[side][m] = make_int4(qx, qy, qz, 0);
            gp[side][m] = make_float4(src[3 * m], src[3 * m + 1], src[3 * m + 2], 0.0f);
            const int c = ((qz >> cshift) * cgy + (qy >> cshift)) * cgx + (qx >> cshift);
            cell_of[m] = c;
            cell_start[side][c + 1] += 1;
        }
        for (int c = 0; c < n_cells; ++c) cell_start[side][c + 1] += cell_start[side][c];
        std::vector<int> fill(cell_start[side].begin(), cell_start[side].end() - 1);
        for (int m = 0; m < d->n_guid; ++m) cell_pts[side][fill[cell_of[m]]++] = m;
    }
    std::vector<int> goff(G + 1, 0);
    std::vector<float4> gsorted[2];
    for (int g = 0; g < G; ++g) goff[g + 1] = goff[g] + gcount[g];
    for (int side = 0; side < 2; ++side) {
        gsorted[side].resize(std::max(d->n_guid, 1));
        std::vector<int> fill(goff.begin(), goff.end() - 1);
        for (int m = 0; m < d->n_guid; ++m) {
            const int g = d->guid_group ? d->guid_group[m] : 0;
            gsorted[side][fill[g]++] = gp[side][m];
        }
    }

    // ---- allocation ----
    morea_problem *p = new (std::nothrow) morea_problem();
    if (!p) return MOREA_ENOMEM;
    cudaGetDevice(&p->device);
    p->V = V;
    p->T = T;
    p->G = G;
    p->max_sol = max_sol;
    p->max_req = max_req;
    p->max_changed = max_changed;
    p->max_star = max_star;
    p->cap_entries = (int)cap;
    p->r = r;
    cudaStream_t st = (cudaStream_t)stream;
    DevProblem &hp = p->hp;
    hp.nx = nx;
    hp.ny = ny;
    hp.nz = nz;
    hp.dtype = d->dtype;
    hp.kbits = k;
    hp.S = S;
    hp.H = H;
    hp.h_mode = d->h_mode;
    hp.g_mode = d->g_mode;
    hp.estimator = d->estimator;
    hp.rate = d->sampling_rate > 0.0f ? d->sampling_rate : 1.0f;
    hp.G = G;
    hp.n_points = V;
    hp.n_tets = T;
    hp.r = (float)r;
    hp.inv_r = (float)(1.0 / r);
    hp.n_guid = d->n_guid;
    hp.cshift = cshift;
    for (int g = 0; g < kMaxGroups; ++g) hp.wgt[g] = wgt[g];
    hp.cgx = cgx;
    hp.cgy = cgy;
    hp.cgz = cgz;
    hp.max_sol = max_sol;

    const size_t esz = d->dtype == MOREA_F16 ? 2 : 4;
    cudaError_t e = cudaSuccess;
    void *img[2] = {nullptr, nullptr};
    int4 *dtets = nullptr, *gq_d[2] = {nullptr, nullptr}, *slot_q = nullptr;
    float *dcd = nullptr, *dmap[2] = {nullptr, nullptr};
    float4 *gp_d[2] = {nullptr, nullptr}, *gsort_d = nullptr;
    uint8_t *band[2] = {nullptr, nullptr};
    unsigned char *quad[2] = {nullptr, nullptr};
    short2 *bandrow[2] = {nullptr, nullptr};
    int *cs_d[2] = {nullptr, nullptr}, *cp_d[2] = {nullptr, nullptr}, *goff_d = nullptr;
    morea_tet_record *cache = nullptr;
    morea_totals *totals = nullptr;
    unsigned *status = nullptr;
    const bool continuous = d->g_mode == MOREA_G_CONTINUOUS;
    const bool sampled = d->estimator == MOREA_EST_SAMPLED;
    const bool banded = continuous && !sampled;          // band rows and their lists (voxel estimator)
    uint8_t *bandd[2] = {nullptr, nullptr};
#define TRY(x)                                                                                     \
    do {                                                                                           \
        e = (x);                                                                                   \
        if (e != cudaSuccess) goto fail;                                                           \
    } while (0)
    for (int s = 0; s < 2; ++s) {
        void *m = nullptr;
        TRY(cudaMalloc(&m, (size_t)N * esz));
        p->allocs.push_back(m);
        img[s] = m;
    }
    TRY(dalloc(p, &dtets, T));
    TRY(dalloc(p, &dcd, T));
    TRY(dalloc(p, &p->v2t_off, V + 1));
    TRY(dalloc(p, &p->v2t_idx, v2t_idx.size()));
    for (int s = 0; s < 2; ++s) {
        TRY(dalloc(p, &gq_d[s], gq[s].size()));
        TRY(dalloc(p, &gp_d[s], gp[s].size()));
        TRY(dalloc(p, &cs_d[s], cell_start[s].size()));
        TRY(dalloc(p, &cp_d[s], cell_pts[s].size()));
        TRY(dalloc(p, &quad[s], (size_t)quad_cells(nx, ny, nz) * esz * 4));
        if (continuous) {
            TRY(dalloc(p, &band[s], (size_t)N));
            if (banded) TRY(dalloc(p, &bandrow[s], (size_t)ny * nz));
            if (G > 0) TRY(dalloc(p, &dmap[s], (size_t)N * G));
            if (sampled && G > 0) TRY(dalloc(p, &bandd[s], (size_t)N));
        }
    }
    TRY(dalloc(p, &goff_d, goff.size()));
    TRY(dalloc(p, &gsort_d, std::max<size_t>(1, (size_t)d->n_guid)));
    TRY(dalloc(p, &slot_q, (size_t)max_sol * 2 * V));
    TRY(dalloc(p, &cache, (size_t)max_sol * T));
    TRY(dalloc(p, &totals, (size_t)max_sol));
    TRY(dalloc(p, &status, 1));
    TRY(dalloc(p, &p->entries, (size_t)cap));
    TRY(dalloc(p, &p->setup, 2 * (size_t)cap));
    TRY(dalloc(p, &p->rout, 2 * (size_t)cap));
    if (banded) TRY(dalloc(p, &p->bandrows, 2 * (size_t)cap * kBandRowsPerItem));
    TRY(dalloc(p, &p->tout, (size_t)cap));
    TRY(dalloc(p, &p->counter, 1));
    TRY(dalloc(p, &p->rinfo, (size_t)max_req));
    TRY(dalloc(p, &p->req_delta, (size_t)max_req));
    TRY(dalloc(p, &p->req_chg_pts, (size_t)max_req * max_changed));
    TRY(dalloc(p, &p->req_chg_q, 2 * (size_t)max_req * max_changed));
    TRY(dalloc(p, &p->dp, 1));
    TRY(dalloc(p, &p->visits, 1));
    TRY(dalloc(p, &p->queue, queue_ints(cap, banded)));

    hp.img[0] = img[0];
    hp.img[1] = img[1];
    hp.dmap[0] = dmap[0];
    hp.dmap[1] = dmap[1];
    hp.band[0] = band[0];
    hp.band[1] = band[1];
    hp.quad[0] = quad[0] + quad_origin(nx, ny) * esz * 4;
    hp.quad[1] = quad[1] + quad_origin(nx, ny) * esz * 4;
    hp.bandrow[0] = bandrow[0];
    hp.bandrow[1] = bandrow[1];
    hp.bandd[0] = bandd[0];
    hp.bandd[1] = bandd[1];
    hp.tets = dtets;
    hp.cdelta = dcd;
    for (int s = 0; s < 2; ++s) {
        hp.gq[s] = gq_d[s];
        hp.gp[s] = gp_d[s];
        hp.cell_start[s] = cs_d[s];
        hp.cell_pts[s] = cp_d[s];
    }
    hp.slot_q = slot_q;
    hp.cache = cache;
    hp.totals = totals;
    hp.status = status;

    // ---- copies and set-up kernels ----
    TRY(cudaMemcpyAsync(img[0], d->image_s, (size_t)N * esz, cudaMemcpyDefault, st));
    TRY(cudaMemcpyAsync(img[1], d->image_t, (size_t)N * esz, cudaMemcpyDefault, st));
    TRY(cudaMemcpyAsync(dtets, tets.data(), sizeof(int4) * T, cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(dcd, cdelta.data(), sizeof(float) * T, cudaMemcpyHostToDevice, st));
    if (d->tissue_mask) {
        // elasticity from mask overlap (App. A.1): staged inputs, freed before returning
        std::vector<int4> q4(V);
        for (int v = 0; v < V; ++v) q4[v] = make_int4(qref[3 * v], qref[3 * v + 1], qref[3 * v + 2], 0);
        uint8_t *dmask = nullptr;
        int4 *dq = nullptr;
        double *dfac = nullptr;
        cudaError_t e = cudaMalloc(&dmask, (size_t)N);
        if (e == cudaSuccess) e = cudaMalloc(&dq, sizeof(int4) * V);
        if (e == cudaSuccess) e = cudaMalloc(&dfac, sizeof(double) * d->n_labels);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dmask, d->tissue_mask, (size_t)N, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dq, q4.data(), sizeof(int4) * V, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dfac, d->tissue_factor, sizeof(double) * d->n_labels, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = launch_tissue_factors(hp, dtets, dq, dmask, dfac, d->n_labels, dcd, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(dmask);
        cudaFree(dq);
        cudaFree(dfac);
        TRY(e);
    }
    TRY(cudaMemcpyAsync(p->v2t_off, v2t_off.data(), sizeof(int) * (V + 1), cudaMemcpyHostToDevice, st));
    if (!v2t_idx.empty())
        TRY(cudaMemcpyAsync(p->v2t_idx, v2t_idx.data(), sizeof(int) * v2t_idx.size(), cudaMemcpyHostToDevice, st));
    for (int s = 0; s < 2; ++s) {
        TRY(cudaMemcpyAsync(gq_d[s], gq[s].data(), sizeof(int4) * gq[s].size(), cudaMemcpyHostToDevice, st));
        TRY(cudaMemcpyAsync(gp_d[s], gp[s].data(), sizeof(float4) * gp[s].size(), cudaMemcpyHostToDevice, st));
        TRY(cudaMemcpyAsync(cs_d[s], cell_start[s].data(), sizeof(int) * cell_start[s].size(),
                            cudaMemcpyHostToDevice, st));
        TRY(cudaMemcpyAsync(cp_d[s], cell_pts[s].data(), sizeof(int) * cell_pts[s].size(),
                            cudaMemcpyHostToDevice, st));
        if (continuous) TRY(cudaMemsetAsync(band[s], 0, (size_t)N, st));
    }
    TRY(cudaMemcpyAsync(goff_d, goff.data(), sizeof(int) * goff.size(), cudaMemcpyHostToDevice, st));
    TRY(cudaMemsetAsync(slot_q, 0, sizeof(int4) * (size_t)max_sol * 2 * V, st));
    TRY(cudaMemsetAsync(cache, 0, sizeof(morea_tet_record) * (size_t)max_sol * T, st));
    TRY(cudaMemsetAsync(totals, 0, sizeof(morea_totals) * (size_t)max_sol, st));
    TRY(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
    TRY(cudaMemsetAsync(p->counter, 0, sizeof(int), st));
    TRY(cudaMemsetAsync(p->entries, 0, sizeof(WorkEntry) * (size_t)cap, st));
    TRY(cudaMemsetAsync(p->setup, 0, sizeof(RasterSetup) * 2 * (size_t)cap, st));
    TRY(cudaMemsetAsync(p->rinfo, 0, sizeof(ReqInfo) * (size_t)max_req, st));
    TRY(cudaMemcpyAsync(p->dp, &hp, sizeof(DevProblem), cudaMemcpyHostToDevice, st));
    for (int s = 0; s < 2; ++s) TRY(launch_build_quads(hp, s, quad[s], st));
    if (continuous && G > 0) {
        for (int s = 0; s < 2; ++s) {
            TRY(cudaMemcpyAsync(gsort_d, gsorted[s].data(), sizeof(float4) * gsorted[s].size(),
                                cudaMemcpyHostToDevice, st));
            TRY(launch_distance_maps(hp, gsort_d, goff_d, dmap[s], band[s], st));
            TRY(cudaStreamSynchronize(st));   // gsort_d is reused for the other side
            if (sampled) TRY(launch_band_dilate(hp, band[s], bandd[s], st));
        }
    }
    if (sampled) TRY(sample_setup(st));
    if (banded) {
        for (int s = 0; s < 2; ++s) TRY(launch_band_rows(hp, s, bandrow[s], st));
        // per-row sorted lists of band voxels (built on the host from the masks)
        std::vector<uint8_t> hband((size_t)N);
        for (int s = 0; s < 2; ++s) {
            TRY(cudaMemcpyAsync(hband.data(), band[s], (size_t)N, cudaMemcpyDeviceToHost, st));
            TRY(cudaStreamSynchronize(st));
            std::vector<int> start((size_t)ny * nz + 1, 0);
            std::vector<int2> recs;
            std::vector<short> rank((size_t)N);
            for (long long row = 0; row < (long long)ny * nz; ++row) {
                const uint8_t *b = hband.data() + row * nx;
                short before = 0;
                for (int x = 0; x < nx; ++x) {
                    rank[(size_t)row * nx + x] = before;
                    if (b[x]) {
                        recs.push_back(make_int2(x | ((int)b[x] << 16), 0));
                        ++before;
                    }
                }
                start[row + 1] = (int)recs.size();
            }
            int *bs = nullptr;
            int2 *brc = nullptr;
            short *brk = nullptr;
            TRY(dalloc(p, &bs, start.size()));
            TRY(dalloc(p, &brc, std::max<size_t>(recs.size(), 1)));
            TRY(dalloc(p, &brk, (size_t)N));
            TRY(cudaMemcpyAsync(bs, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice, st));
            if (!recs.empty())
                TRY(cudaMemcpyAsync(brc, recs.data(), sizeof(int2) * recs.size(), cudaMemcpyHostToDevice, st));
            TRY(cudaMemcpyAsync(brk, rank.data(), sizeof(short) * (size_t)N, cudaMemcpyHostToDevice, st));
            hp.band_start[s] = bs;
            hp.band_rec[s] = brc;
            hp.band_rank[s] = brk;
            TRY(launch_band_records(hp, s, brc, st));
            TRY(cudaStreamSynchronize(st));
        }
        TRY(cudaMemcpyAsync(p->dp, &hp, sizeof(DevProblem), cudaMemcpyHostToDevice, st));
    }
    TRY(cudaStreamSynchronize(st));
#undef TRY
    *out = p;
    return MOREA_OK;
fail:
    cudaStreamSynchronize(st);
    cudaGetLastError();
    morea_destroy_problem(p);
    return e == cudaErrorMemoryAllocation ? MOREA_ENOMEM : MOREA_ECUDA;
}

morea_status morea_eval_full(morea_problem *p, int32_t n_sol, const int32_t *slot, const float *src_pts,
                             const float *tgt_pts, double *obj, uint8_t *folded, double *severity,
                             void *stream)
{
    if (!p || n_sol < 1 || n_sol > p->max_sol || !src_pts || !tgt_pts || !obj || !folded) return MOREA_EINVAL;
    DeviceGuard g(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = launch_snap_slots(p->dp, p->hp, n_sol, slot, src_pts, tgt_pts, (int4 *)p->hp.slot_q,
                                      p->max_sol, st);
    if (e == cudaSuccess)
        e = launch_full_entries(p->dp, p->hp, n_sol, slot, p->entries, p->setup, p->tout, st);
    if (e == cudaSuccess) {
        const long long items = 2LL * n_sol * p->T;
        const int grid = (int)std::min<long long>((long long)sm_count() * p->launch.blocks_per_sm, (items + 7) / 8);
        e = timed_raster(p, nullptr, n_sol * p->T, grid, false, st);
    }
    if (e == cudaSuccess)
        e = launch_reduce_full(p->dp, p->hp, n_sol, slot, p->tout, p->rout, obj, folded, severity, st);
    return from_cuda(e);
}

morea_status morea_eval_partial(morea_problem *p, int32_t n_req, const int32_t *slot, const int32_t *chg_off,
                                const int32_t *chg_pts, const float *chg_src, const float *chg_tgt, double *obj,
                                uint8_t *folded, double *severity, const uint8_t *commit, void *stream)
{
    if (!p || n_req < 1 || n_req > p->max_req || !slot || !chg_off || !chg_pts || !chg_src || !chg_tgt || !obj ||
        !folded)
        return MOREA_EINVAL;
    DeviceGuard g(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(p->counter, 0, sizeof(int), st);
    // the entry pass orders the image pass's items (largest copies first): its counters start at zero
    if (e == cudaSuccess) e = cudaMemsetAsync(p->queue, 0, kQueueList * sizeof(int), st);
    if (e == cudaSuccess)
        e = launch_partial_entries(p->dp, p->hp, n_req, slot, chg_off, chg_pts, chg_src, chg_tgt, p->max_sol,
                                   p->max_changed, p->v2t_off, p->v2t_idx, p->entries, p->setup, p->tout,
                                   p->cap_entries, p->counter, p->rinfo, p->req_chg_pts, p->req_chg_q, p->queue,
                                   st);
    if (e == cudaSuccess)
        e = timed_raster(p, p->counter, p->cap_entries, sm_count() * p->launch.blocks_per_sm, true, st);
    if (e == cudaSuccess)
        e = launch_partial_finalize(p->dp, p->hp, n_req, p->rinfo, p->entries, p->tout, p->rout, p->req_delta, obj,
                                    folded, severity, st);
    if (e == cudaSuccess) p->last_nreq = n_req;
    if (e == cudaSuccess && commit)
        e = launch_partial_commit(p->dp, p->hp, n_req, commit, p->rinfo, p->entries, p->tout, p->rout,
                                  p->req_delta, p->req_chg_pts, p->req_chg_q, p->max_changed, p->counter,
                                  p->cap_entries, (int4 *)p->hp.slot_q, st);
    return from_cuda(e);
}

morea_status morea_commit_partial(morea_problem *p, int32_t n_req, const uint8_t *accept, void *stream)
{
    if (!p || !accept || n_req < 1 || n_req != p->last_nreq) return MOREA_EINVAL;
    DeviceGuard g(p->device);
    return from_cuda(launch_partial_commit(p->dp, p->hp, n_req, accept, p->rinfo, p->entries, p->tout, p->rout,
                                           p->req_delta, p->req_chg_pts, p->req_chg_q, p->max_changed,
                                           p->counter, p->cap_entries, (int4 *)p->hp.slot_q,
                                           (cudaStream_t)stream));
}

morea_status morea_displacement(morea_problem *p, const float *src, const float *tgt, int32_t side, float *dvf,
                                const uint8_t *labels_own, const uint8_t *labels_other, int32_t n_labels,
                                int64_t *overlap, void *stream)
{
    if (!p || !src || !tgt || (side != 0 && side != 1)) return MOREA_EINVAL;
    const bool labels = labels_own || labels_other || overlap;
    if (labels && (!labels_own || !labels_other || !overlap || n_labels < 1 || n_labels > dvf_max_labels()))
        return MOREA_EINVAL;
    DeviceGuard g(p->device);
    return from_cuda(launch_dvf(p->dp, p->hp, src, tgt, side, dvf, labels ? labels_own : nullptr,
                                labels ? labels_other : nullptr, labels ? n_labels : 0,
                                labels ? reinterpret_cast<unsigned long long *>(overlap) : nullptr, nullptr,
                                (cudaStream_t)stream));
}

morea_status morea_warp_labels(morea_problem *p, const float *src, const float *tgt, int32_t side,
                               const uint8_t *labels_other, uint8_t *warped, void *stream)
{
    if (!p || !src || !tgt || (side != 0 && side != 1) || !labels_other || !warped) return MOREA_EINVAL;
    DeviceGuard g(p->device);
    return from_cuda(launch_dvf(p->dp, p->hp, src, tgt, side, nullptr, nullptr, labels_other, 0, nullptr, warped,
                                (cudaStream_t)stream));
}

morea_status morea_slot_objectives(morea_problem *p, int32_t n_sol, const int32_t *slot, double *obj,
                                   uint8_t *folded, double *severity, void *stream)
{
    if (!p || n_sol < 1 || !obj || !folded) return MOREA_EINVAL;
    DeviceGuard g(p->device);
    return from_cuda(launch_slot_objectives(p->dp, n_sol, slot, obj, folded, severity, (cudaStream_t)stream));
}

size_t morea_sample_elements_workspace(int32_t n_clusters, int32_t n_elements)
{
    if (n_clusters < 1 || n_elements < 1) return 0;
    return sample_elements_bytes(n_clusters, n_elements);
}

morea_status morea_sample_elements(morea_problem *p, int32_t n_pop, const float *src, const float *tgt,
                                   int32_t n_clusters, int32_t cluster_size, const int32_t *members,
                                   int32_t n_elements, const int32_t *elements, const uint8_t *fixed,
                                   const float *cmult, int32_t n_req, const int32_t *req_sol,
                                   const int32_t *req_cluster, const int32_t *req_element, const float *z,
                                   void *work, size_t work_bytes, float *new_src, float *new_tgt, void *stream)
{
    if (!p || n_pop < 1 || !src || !tgt || n_clusters < 1 || cluster_size < 1 || !members || n_elements < 1 ||
        !elements || !cmult || n_req < 0 || !work)
        return MOREA_EINVAL;
    if (n_req > 0 && (!req_sol || !req_cluster || !req_element || !z || !new_src || !new_tgt)) return MOREA_EINVAL;
    if ((reinterpret_cast<uintptr_t>(elements) & 7) != 0 || (reinterpret_cast<uintptr_t>(work) & 15) != 0)
        return MOREA_EINVAL;
    if (work_bytes < sample_elements_bytes(n_clusters, n_elements)) return MOREA_EINVAL;
    DeviceGuard g(p->device);
    return from_cuda(launch_sample_elements(p->V, n_pop, src, tgt, n_clusters, cluster_size, members, n_elements,
                                            elements, fixed, cmult, n_req, req_sol, req_cluster, req_element, z,
                                            work, new_src, new_tgt, (cudaStream_t)stream));
}

morea_status morea_init_noise(morea_problem *p, int32_t n_sol, float *src, float *tgt, const uint8_t *fixed,
                              int32_t n_kernels, const float *kernels, int32_t max_rounds, int32_t *rounds,
                              void *stream)
{
    if (!p || n_sol < 1 || n_sol > (1 << 29) || !src || !tgt || n_kernels < 0 || (n_kernels > 0 && !kernels) ||
        max_rounds < 0 || !rounds)
        return MOREA_EINVAL;
    if (init_smem_bytes(p->V, n_kernels) > 200 * 1024) return MOREA_EINVAL;
    DeviceGuard g(p->device);
    return from_cuda(launch_init(p->dp, p->hp, n_sol, src, tgt, fixed, n_kernels, kernels, max_rounds, rounds,
                                 (cudaStream_t)stream));
}

morea_status morea_repair_folds(morea_problem *p, int32_t n_sol, float *src, float *tgt, const float *noise,
                                int32_t max_points, float scale, const uint8_t *fixed, int32_t *moved,
                                double *severity, void *stream)
{
    if (!p || n_sol < 1 || !src || !tgt || !noise || !moved || !severity || max_points < 1 || !(scale > 0.0f) ||
        std::isinf(scale))
        return MOREA_EINVAL;
    if ((size_t)4 * ((p->V + 31) / 32) * sizeof(unsigned) > 200 * 1024) return MOREA_EINVAL;
    DeviceGuard g(p->device);
    return from_cuda(launch_repair(p->dp, p->hp, p->v2t_off, p->v2t_idx, n_sol, src, tgt, noise, max_points,
                                   (double)scale, fixed, moved, severity, (cudaStream_t)stream));
}

morea_status morea_check_folds(morea_problem *p, int32_t n_sol, const float *src_pts, const float *tgt_pts,
                               uint8_t *folded, double *severity, void *stream)
{
    if (!p || n_sol < 1 || !src_pts || !tgt_pts || !folded) return MOREA_EINVAL;
    DeviceGuard g(p->device);
    return from_cuda(launch_check_folds(p->dp, p->hp, n_sol, src_pts, tgt_pts, folded, severity,
                                        (cudaStream_t)stream));
}

morea_status morea_read_records(morea_problem *p, int32_t n_sol, const int32_t *slot, morea_tet_record *out,
                                void *stream)
{
    if (!p || n_sol < 1 || n_sol > p->max_sol || !out) return MOREA_EINVAL;
    DeviceGuard g(p->device);
    return from_cuda(launch_gather_records(p->hp, n_sol, slot, out, (cudaStream_t)stream));
}

morea_status morea_read_totals(morea_problem *p, int32_t n_sol, const int32_t *slot, morea_totals *out,
                               void *stream)
{
    if (!p || n_sol < 1 || n_sol > p->max_sol || !out) return MOREA_EINVAL;
    DeviceGuard g(p->device);
    return from_cuda(launch_gather_totals(p->hp, n_sol, slot, out, (cudaStream_t)stream));
}

morea_status morea_partial_features(morea_problem *p, int32_t n_req, const int32_t *slot, const int32_t *chg_off,
                                    const int32_t *chg_pts, const float *chg_src, const float *chg_tgt, float *out,
                                    void *stream)
{
    if (!p || n_req < 1 || !slot || !chg_off || !out) return MOREA_EINVAL;
    DeviceGuard g(p->device);
    return from_cuda(launch_partial_features(p->dp, n_req, slot, chg_off, chg_pts, chg_src, chg_tgt, out,
                                             (cudaStream_t)stream));
}

morea_status morea_device_status(morea_problem *p, void *stream, uint32_t *bits)
{
    if (!p) return MOREA_EINVAL;
    DeviceGuard g(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned h = 0;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(&h, p->hp.status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(p->hp.status, 0, sizeof(unsigned));
    if (e != cudaSuccess) return MOREA_ECUDA;
    if (bits) *bits = h;
    return h ? MOREA_EDEVICE : MOREA_OK;
}

morea_status morea_profile(morea_problem *p, uint32_t flags)
{
    if (!p || flags > 3u) return MOREA_EINVAL;
    DeviceGuard g(p->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemset(p->visits, 0, sizeof(unsigned long long));
    p->prof = flags;
    p->ev_used = 0;
    return from_cuda(e);
}

morea_status morea_profile_read(morea_problem *p, double *raster_ms, int64_t *launches, int64_t *visits)
{
    if (!p) return MOREA_EINVAL;
    DeviceGuard g(p->device);
    double ms = 0.0;
    for (size_t i = 0; i + 1 < p->ev_used; i += 2) {
        cudaError_t e = cudaEventSynchronize(p->ev[i + 1]);
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p->ev[i], p->ev[i + 1]);
        if (e != cudaSuccess) return MOREA_ECUDA;
        ms += t;
    }
    unsigned long long v = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&v, p->visits, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return MOREA_ECUDA;
    if (raster_ms) *raster_ms = ms;
    if (launches) *launches = (int64_t)(p->ev_used / 2);
    if (visits) *visits = (int64_t)v;
    return MOREA_OK;
}

morea_status morea_problem_info(const morea_problem *p, int32_t *n_points, int32_t *n_tets, int32_t *n_groups,
                                double *trunc_radius, int32_t *subvoxel_bits)
{
    if (!p) return MOREA_EINVAL;
    if (n_points) *n_points = p->V;
    if (n_tets) *n_tets = p->T;
    if (n_groups) *n_groups = p->G;
    if (trunc_radius) *trunc_radius = p->r;
    if (subvoxel_bits) *subvoxel_bits = p->hp.kbits;
    return MOREA_OK;
}

}  // extern "C"
