// The hot loop of libmorea (steps a4-a7): for each (work entry, side) one
// warp walks the voxel-centre rows that can meet the tet copy (per z-slice,
// the y-extent of its cross-section), solves the exact integer x-interval of
// each row, queues the rows' voxels and processes them 32 at a time, one per
// lane: it maps every voxel centre p into the other image with the tet's
// affine map, samples the other image trilinearly, accumulates h (Sec. 4.1.2)
// in compensated FP32, and reduces the per-lane sums with warp shuffles into
// one record per (entry, side).  The continuous guidance term (Sec. 4.1.3)
// is summed by k_guidance over the rows this pass records.
//
// Voxel association (exact): a voxel centre P is inside the copy iff for
// every face f: A_f i + B_f(j, k) > 0 (integers, simulation-of-simplicity tie
// bit folded into B).  Each face bound is first estimated in FP32 and then
// corrected with exact int64 evaluations, so the interval does not depend on
// the estimate's rounding.
//
// Memory traffic per voxel visit: the own voxel (one 4- or 2-byte load), one
// 16- or 8-byte load per z-plane of the other image's 2x2x2 neighbourhood
// from its "quad" copy, and the band mask only in rows that touch a guidance
// band.
#include <algorithm>

#include "image_ops.cuh"

namespace morea {

namespace {

// Pair-transfer guidance of one tet copy: the guidance points of this side
// located in the copy (exact perturbed inside test on their snapped
// coordinates), mapped and compared with their partners.
__device__ __noinline__ void guidance_pairs(const DevProblem &P, const RasterSetup *su, int side, int lane,
                                            float &s_g, float &c_g, int &ngp)
{
    const int cs = P.cshift, kb = P.kbits;
    const int cx0 = max(0, su->qlo[0] >> cs), cx1 = min(P.cgx - 1, su->qhi[0] >> cs);
    const int cy0 = max(0, su->qlo[1] >> cs), cy1 = min(P.cgy - 1, su->qhi[1] >> cs);
    const int cz0 = max(0, su->qlo[2] >> cs), cz1 = min(P.cgz - 1, su->qhi[2] >> cs);
    const float inv_s = 1.0f / (float)P.S;
    const float *M = su->M;
    for (int cz = cz0; cz <= cz1; ++cz)
        for (int cy = cy0; cy <= cy1; ++cy)
            for (int cx = cx0; cx <= cx1; ++cx) {
                const int c = (cz * P.cgy + cy) * P.cgx + cx;
                const int p0 = P.cell_start[side][c], p1 = P.cell_start[side][c + 1];
                for (int p = p0 + lane; p < p1; p += 32) {
                    const int mi = P.cell_pts[side][p];
                    const int4 q = P.gq[side][mi];
                    bool in = true;
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        const long long val = (su->f[f].ax >> kb) * q.x + (su->f[f].by >> kb) * q.y +
                                              (su->f[f].bz >> kb) * q.z + su->ct[f];
                        in = in && val > 0;
                    }
                    if (in) {
                        const float dx = q.x * inv_s - 0.5f - su->s0[0];
                        const float dy = q.y * inv_s - 0.5f - su->s0[1];
                        const float dz = q.z * inv_s - 0.5f - su->s0[2];
                        const float4 go = P.gp[1 - side][mi];
                        const float ex = fmaf(M[0], dx, fmaf(M[1], dy, fmaf(M[2], dz, su->t0[0]))) - go.x;
                        const float ey = fmaf(M[3], dx, fmaf(M[4], dy, fmaf(M[5], dz, su->t0[1]))) - go.y;
                        const float ez = fmaf(M[6], dx, fmaf(M[7], dy, fmaf(M[8], dz, su->t0[2]))) - go.z;
                        kadd(s_g, c_g, fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
                        ngp += 1;
                    }
                }
            }
}

// Pass modes of the image kernel.
constexpr int kPassImage = 0;       // f_intensity only
constexpr int kPassImageBand = 1;   // f_intensity + record the rows that touch a guidance band
constexpr int kPassImagePairs = 2;  // f_intensity + pair-transfer guidance

// Band-row records: per (entry, side) up to kBandRows segments (x range,
// row) of voxels that may lie in a guidance band; k_guidance processes them.
// A count above kBandRows means "overflow: recompute the rows".
constexpr int kBandRows = kBandRowsPerItem;

__device__ __forceinline__ int2 pack_band_row(int lo, int hi, int j, int k)
{
    return make_int2(lo | (hi << 16), j | (k << 16));
}

// Per-warp queue of the rows found by the row phase.  Voxels of successive
// rows form one stream (index u); a row occupies [start, next row's start),
// its voxel x = d + u, its image row starts at linear index base, and
// (rx, ry, rz) holds the row's part of the affine map, so a voxel's mapped
// position is fma(M[a][0], x - s0x, r_a): the same FMA chain as evaluating the
// map from scratch.  Rows accumulate across row batches and the voxels are
// processed in full windows of 32 (one voxel per lane, coalesced along rows).
constexpr int kRowQ = 128;              // ring capacity (rows); power of two
constexpr int kWin = 32;                // voxels per window (one per lane)
struct RowQueue {
    int start[kRowQ];
    int2 db[kRowQ];                      // (d, base)
    float4 r[kRowQ];                     // (rx, ry, rz, -)
    float4 mcol;                         // first column of M and s0.x of the current item
    float4 rowc[3];                      // per map row a: (M[a][1], M[a][2], t0[a], s0.y | s0.z | -)
};

// Image pass (a4, a5, a7): one warp per (entry, side).
template <typename TI, int HMODE, int PASS, bool ORDERED>
__global__ void __launch_bounds__(kBlock, 6) k_raster(const DevProblem *__restrict__ probs,
                                                     const WorkEntry *__restrict__ entries,
                                                     const RasterSetup *__restrict__ setup,
                                                     RasterOut *__restrict__ rout, int2 *__restrict__ bandrows,
                                                     const int *n_entries_dev, int n_entries_host, int chunk,
                                                     int *queue, const int *order, BatchClock *clock)
{
    using QT = typename QuadOf<TI>::T;
    __shared__ RowQueue rowq[kBlock / 32];
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const unsigned upto = lane == 31 ? FULL : ((2u << lane) - 1u);   // bits 0..lane
    RowQueue &Q = rowq[threadIdx.x >> 5];
    const int n_ent = n_entries_dev ? min(*n_entries_dev, n_entries_host) : n_entries_host;
    const int n_items = 2 * n_ent;
    // ORDERED: the large items the entry pass listed first, then every item in
    // its own order except those
    const int n_big = ORDERED ? min(queue[kQueueOrderBig], n_items) : 0;
    run_items(n_big + n_items, chunk, queue + kQueueRaster, [&](const int qi) {
        const int item = qi < n_big ? order[qi] : qi - n_big;
        const int side = item >= n_ent ? 1 : 0;      // all source sides, then all target sides
        const int e = item - side * n_ent;
        const RasterSetup *su = setup + 2 * (size_t)e + side;
        const unsigned char *sb = reinterpret_cast<const unsigned char *>(su);
        const int4 bx = __ldg(reinterpret_cast<const int4 *>(sb + offsetof(RasterSetup, ilo)));
        const int2 bz2 = __ldg(reinterpret_cast<const int2 *>(sb + offsetof(RasterSetup, klo)));
        const int valid = __ldg(reinterpret_cast<const int *>(sb + offsetof(RasterSetup, valid)));
        if (ORDERED && qi >= n_big && (valid & 1) &&
            (long long)max(bx.y - bx.x + 1, 0) * max(bx.w - bx.z + 1, 0) * max(bz2.y - bz2.x + 1, 0) >=
                kBigItemVoxels)
            return;                                   // a large item, done from the list
        float s_img = 0.0f, c_img = 0.0f, s_g = 0.0f, c_g = 0.0f;
        int nvox = 0, ngp = 0;
        int nband = 0;                                // band rows recorded (warp-uniform)
        int2 *brec = PASS == kPassImageBand ? bandrows + (2 * (size_t)e + side) * kBandRows : nullptr;
        if (valid & 1) {
            const DevProblem &P = probs[entries[e].prob];
            const int nx = P.nx, ny = P.ny, nz = P.nz;
            const TI *own = (const TI *)P.img[side];
            const QT *oq = (const QT *)P.quad[1 - side];
            const int ilo = bx.x, ihi = bx.y, jlo = bx.z, klo = bz2.x;
            const int nyb = max(bx.w - jlo + 1, 1), nzb = bz2.y - klo + 1;
            const int n_rows = (ilo <= ihi && bx.w >= jlo && nzb > 0) ? nyb * nzb : 0;
            const bool inner = (valid & 2) != 0;
            if (lane == 0) {
                // M = (a.x a.y a.z; a.w b.x b.y; b.z b.w c.x), s0 = c.yzw, t0 = t.xyz
                const float4 ma = __ldg(reinterpret_cast<const float4 *>(sb + offsetof(RasterSetup, M)));
                const float4 mb = __ldg(reinterpret_cast<const float4 *>(sb + offsetof(RasterSetup, M) + 16));
                const float4 mc = __ldg(reinterpret_cast<const float4 *>(sb + offsetof(RasterSetup, M) + 32));
                const float4 mt = __ldg(reinterpret_cast<const float4 *>(sb + offsetof(RasterSetup, t0)));
                Q.mcol = make_float4(ma.x, ma.w, mb.z, mc.y);
                Q.rowc[0] = make_float4(ma.y, ma.z, mt.x, mc.z);
                Q.rowc[1] = make_float4(mb.x, mb.y, mt.y, mc.w);
                Q.rowc[2] = make_float4(mb.w, mc.x, mt.z, 0.0f);
            }
            __syncwarp();
            // row queue state (warp-uniform): live rows [head, tail), voxel
            // stream [pend, total) not yet processed
            int head = 0, tail = 0, pend = 0, total = 0;
            auto voxel = [&](int u, int d, int base, float rx, float ry, float rz, float M00, float M10, float M20,
                             float s0x) {
                const int x = d + u;
                const float a = ld_img(own, base + x);
                const float dx = (float)x - s0x;
                const float yx = fmaf(M00, dx, rx);
                const float yy = fmaf(M10, dx, ry);
                const float yz = fmaf(M20, dx, rz);
                const float b = inner ? trilin_quad_inner(oq, nx + 1, (nx + 1) * (ny + 1), yx, yy, yz)
                                      : trilin_quad(oq, nx, ny, nz, yx, yy, yz);
                kadd(s_img, c_img, hfun<HMODE>(a, b));
            };
            // voxels [wbase, wbase + w) of the stream, one per lane.  `head` is
            // the last row starting at or before wbase (a row that starts
            // exactly at wbase may follow it when it was appended after the
            // previous window); the later rows that start inside the window
            // set bit (start - wbase) of `starts`, so a lane's row is
            // head + popc(starts & bits <= its position).  The return value
            // counts the rows starting at or before wbase + 32: how far
            // `head` moves for the next full window.
            auto window = [&](int wbase, int w) -> int {
                const int r = head + 1 + lane;
                unsigned bit = 0u;
                int st = 0x7fffffff;
                if (r < tail) {
                    st = Q.start[r & (kRowQ - 1)];
                    if (st < wbase + 32) bit = 1u << (st - wbase);
                }
                const unsigned starts = __reduce_or_sync(FULL, bit);
                const unsigned done = __ballot_sync(FULL, st <= wbase + 32);
                const int q = (head + __popc(starts & upto)) & (kRowQ - 1);
                if (lane < w) {
                    const int2 db = Q.db[q];
                    const float4 r = Q.r[q];
                    const float4 mc = Q.mcol;
                    voxel(wbase + lane, db.x, db.y, r.x, r.y, r.z, mc.x, mc.y, mc.z, mc.w);
                }
                __syncwarp();
                return __popc(done);
            };
            // The 64 voxels [wbase, wbase + 64), two per lane: wbase + lane,
            // then wbase + 32 + lane, the order of two 32-voxel windows, so the
            // lane sums are the same.  Both halves' loads can be in flight at
            // once.  It needs the 32 rows after head to hold every row that
            // starts in the span (the 32nd of them starts at or after
            // wbase + 64, or there is none); otherwise it returns -1 and does
            // nothing.  The rows starting in the first half set bit
            // (start - wbase) of `lo`, those in the second half bit
            // (start - wbase - 32) of `hi`.
            auto window2 = [&](int wbase) -> int {
                const int r = head + 1 + lane;
                int st = 0x7fffffff;
                if (r < tail) st = Q.start[r & (kRowQ - 1)];
                if (__shfl_sync(FULL, st, 31) < wbase + 2 * kWin) return -1;
                const int rel = st - wbase;
                const unsigned lo = __reduce_or_sync(FULL, rel < kWin ? 1u << rel : 0u);
                const unsigned hi = __reduce_or_sync(FULL, rel >= kWin && rel < 2 * kWin ? 1u << (rel - kWin) : 0u);
                const unsigned done = __ballot_sync(FULL, st <= wbase + 2 * kWin);
                const int q0 = (head + __popc(lo & upto)) & (kRowQ - 1);
                const int q1 = (head + __popc(lo) + __popc(hi & upto)) & (kRowQ - 1);
                {
                    const int2 db = Q.db[q0];
                    const float4 rq = Q.r[q0];
                    const float4 mc = Q.mcol;
                    voxel(wbase + lane, db.x, db.y, rq.x, rq.y, rq.z, mc.x, mc.y, mc.z, mc.w);
                }
                {
                    const int2 db = Q.db[q1];
                    const float4 rq = Q.r[q1];
                    const float4 mc = Q.mcol;
                    voxel(wbase + kWin + lane, db.x, db.y, rq.x, rq.y, rq.z, mc.x, mc.y, mc.z, mc.w);
                }
                __syncwarp();
                return __popc(done);
            };
            // Rows of the bounding box that can meet the copy, 32 z-slices at
            // a time: lane l finds the y-extent [jl, jl + ns) of slice
            // klo + kc + l, a warp scan numbers the rows of the chunk, and the
            // row of lane l in batch rb is found by a binary search over the
            // scan.  row_interval stays the exact test of every row.
            const float Sf = (float)P.S, Hf = (float)P.H;
            for (int kc = 0; kc < nzb && n_rows > 0; kc += 32) {
                int jl = 0, ns = 0;
                if (kc + lane < nzb) {
                    float y0, y1;
                    slice_y_extent(entries[e].q[side], (float)(klo + kc + lane) * Sf + Hf, y0, y1);
                    if (y0 <= y1) {
                        const float m = Sf * 0.0625f + 1.0f;   // 1/16 voxel + 1 unit
                        jl = max(jlo, (int)ceilf((y0 - m - Hf) / Sf));
                        ns = max(0, min(bx.w, (int)floorf((y1 + m - Hf) / Sf)) - jl + 1);
                    }
                }
                int srow = ns;                            // inclusive scan of the slices' row counts
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(FULL, srow, o);
                    if (lane >= o) srow += v;
                }
                const int chunk_rows = __shfl_sync(FULL, srow, 31);
                for (int rb = 0; rb < chunk_rows; rb += 32) {
                    const int r = rb + lane;
                    int sl = 0;                           // first slice whose scan exceeds r
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const int v = __shfl_sync(FULL, srow, sl + o - 1);
                        if (v <= r) sl += o;
                    }
                    const int s_end = __shfl_sync(FULL, srow, sl);
                    const int s_n = __shfl_sync(FULL, ns, sl);
                    const int s_jl = __shfl_sync(FULL, jl, sl);
                    const int dk = kc + sl;
                    const int j = s_jl + r - (s_end - s_n), k = klo + dk;
                    const int dj = j - jlo;
                    int lo = 1, hi = 0;
                    if (r < chunk_rows) row_interval(su->f, dj, dk, ilo, ihi, lo, hi);
                    if (PASS == kPassImageBand) {
                        // record the band part of each row (warp-aggregated append)
                        int blo = 1, bhi = 0;
                        if (hi >= lo) {
                            const short2 br = __ldg(P.bandrow[side] + (k * ny + j));
                            blo = max(lo, (int)br.x);
                            bhi = min(hi, (int)br.y);
                        }
                        const bool band = blo <= bhi;
                        const unsigned bm = __ballot_sync(FULL, band);
                        if (bm) {
                            const int pos = nband + __popc(bm & ((1u << lane) - 1u));
                            if (band && pos < kBandRows) brec[pos] = pack_band_row(blo, bhi, j, k);
                            nband += __popc(bm);
                        }
                    }
                    const int cnt = max(0, hi - lo + 1);
                    int incl = cnt;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int v = __shfl_up_sync(FULL, incl, o);
                        if (lane >= o) incl += v;
                    }
                    const int batch_total = __shfl_sync(FULL, incl, 31);
                    nvox += batch_total;
                    // append the non-empty rows to the queue
                    const unsigned ne = __ballot_sync(FULL, cnt > 0);
                    if (cnt > 0) {
                        // the row's part of the map: r_a = M[a][1] dy + M[a][2] dz + t0[a]
                        const float4 c0 = Q.rowc[0], c1 = Q.rowc[1], c2 = Q.rowc[2];
                        const int q = (tail + __popc(ne & lt_mask)) & (kRowQ - 1);
                        const int st = total + incl - cnt;
                        const float dy = (float)j - c0.w, dz = (float)k - c1.w;
                        Q.start[q] = st;
                        Q.db[q] = make_int2(lo - st, (k * ny + j) * nx);
                        Q.r[q] = make_float4(fmaf(c0.x, dy, fmaf(c0.y, dz, c0.z)), fmaf(c1.x, dy, fmaf(c1.y, dz, c1.z)),
                                             fmaf(c2.x, dy, fmaf(c2.y, dz, c2.z)), 0.0f);
                    }
                    tail += __popc(ne);
                    total += batch_total;
                    __syncwarp();
                    while (total - pend >= kWin) {
                        if (total - pend >= 2 * kWin) {
                            const int adv = window2(pend);
                            if (adv >= 0) {
                                head += adv;
                                pend += 2 * kWin;
                                continue;
                            }
                        }
                        head += window(pend, kWin);
                        pend += kWin;
                    }
                }
            }
            if (total > pend) window(pend, total - pend);
            __syncwarp();
            if (PASS == kPassImagePairs && P.n_guid > 0) guidance_pairs(P, su, side, lane, s_g, c_g, ngp);
        }
        const float e_img = warp_comp_sum(s_img, -c_img);
        float e_g = 0.0f;
        if (PASS == kPassImagePairs) {
            e_g = warp_comp_sum(s_g, -c_g);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ngp += __shfl_xor_sync(FULL, ngp, o);
        }
        if (PASS == kPassImageBand) ngp = nband;      // band rows for k_guidance (cleared there)
        if (lane == 0) {
            RasterOut ro;
            ro.e_img = e_img;
            ro.e_guid = e_g;
            ro.n_vox = nvox;
            ro.n_gp = ngp;
            rout[2 * (size_t)e + side] = ro;
            if (PASS == kPassImageBand && nband > 0) queue[kQueueList + atomicAdd(queue + kQueueListCount, 1)] = item;
            if (clock) {                              // batched evaluation: completion of the problem's items
                const int pi = entries[e].prob;
                if (PASS == kPassImageBand && nband > 0) atomicAdd(&clock->guid_total[pi], 1);
                if (atomicAdd(&clock->raster_done[pi], 1) + 1 == clock->raster_total[pi])
                    clock->t_raster[pi] = global_ns();
            }
        }
    });
}

// Continuous guidance term of one band voxel, in two parts so that a lane
// can load the samples of several voxels before it sums any of them.
// band_load maps the voxel x of row (j, k) = (ojk & 0xffff, ojk >> 16),
// whose band record is r, by the copy's affine map (M = m0.xyz / m0.w m1.xy
// / m1.zw m2.x, s0 = m2.yzw, t0 = t4.xyz) and samples the other side's
// distance map of the lowest band group; band_sum adds that group's term and
// then the terms of the voxel's other groups, lowest first.
struct BandVoxel {
    int idx;                              // voxel index in the own image
    unsigned mk;                          // band groups still to add (lowest first)
    float av, dv;                         // own distance and sampled distance of the lowest group
    float yx, yy, yz;                     // mapped position
};

__device__ __forceinline__ BandVoxel band_load(const DevProblem &P, int side, float4 m0, float4 m1, float4 m2,
                                               float4 t4, int2 r, int ojk)
{
    BandVoxel b;
    const int x = r.x & 0xffff;
    const int oj = ojk & 0xffff, okk = ojk >> 16;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    b.idx = (okk * ny + oj) * nx + x;
    const float dx = (float)x - m2.y, dy = (float)oj - m2.z, dz = (float)okk - m2.w;
    b.yx = fmaf(m0.x, dx, fmaf(m0.y, dy, fmaf(m0.z, dz, t4.x)));
    b.yy = fmaf(m0.w, dx, fmaf(m1.x, dy, fmaf(m1.y, dz, t4.y)));
    b.yz = fmaf(m1.z, dx, fmaf(m1.w, dy, fmaf(m2.x, dz, t4.z)));
    b.mk = (unsigned)r.x >> 16;
    b.av = __int_as_float(r.y);
    const int g = __ffs(b.mk) - 1;
    b.dv = trilin_plain(P.dmap[1 - side] + (size_t)g * ((size_t)nx * ny * nz), nx, ny, nz, b.yx, b.yy, b.yz);
    return b;
}

__device__ __forceinline__ void band_sum(const DevProblem &P, int side, BandVoxel b, float &s_g, float &c_g)
{
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const size_t n_vox = (size_t)nx * ny * nz;
    unsigned mk = b.mk;
    float av = b.av, dv = b.dv;
    while (mk) {
        const int g = __ffs(mk) - 1;
        mk &= mk - 1;
        if (av < P.r) {
            const float w = P.wgt[g] * (P.r - av) * P.inv_r;
            const float df = av - dv;
            kadd(s_g, c_g, w * df * df);
        }
        if (mk) {
            const size_t off = (size_t)(__ffs(mk) - 1) * n_vox;
            av = __ldg(P.dmap[side] + off + b.idx);
            dv = trilin_plain(P.dmap[1 - side] + off, nx, ny, nz, b.yx, b.yy, b.yz);
        }
    }
}

// Continuous guidance (a6): for every (entry, side) that the image pass listed
// as having band rows, the band voxels of those rows (rows recorded by the image pass, or recomputed when
// there were more than kBandRows; band voxels from the per-row sorted
// list); writes e_guid and clears the count.  Mapped positions use the same
// FP32 affine map as the image pass.
__global__ void __launch_bounds__(kBlock, 4) k_guidance(const DevProblem *__restrict__ probs,
                                                       const WorkEntry *__restrict__ entries,
                                                       const RasterSetup *__restrict__ setup,
                                                       RasterOut *__restrict__ rout,
                                                       const int2 *__restrict__ bandrows, const int *n_entries_dev,
                                                       int n_entries_host, int chunk, int *queue)
{
    const int lane = threadIdx.x & 31;
    const int n_ent = n_entries_dev ? min(*n_entries_dev, n_entries_host) : n_entries_host;
    const int n_list = min(queue[kQueueListCount], 2 * n_ent);
    const int *list = queue + kQueueList;
    run_items(n_list, chunk, queue + kQueueGuidance, [&](const int li) {
        const int item = list[li];
        const int side = item >= n_ent ? 1 : 0;
        const int e = item - side * n_ent;
        RasterOut *ro = rout + 2 * (size_t)e + side;
        const int nband = ro->n_gp;                   // warp-uniform, > 0 for listed items
        const RasterSetup *su = setup + 2 * (size_t)e + side;
        const unsigned char *sb = reinterpret_cast<const unsigned char *>(su);
        const float4 m0 = __ldg(reinterpret_cast<const float4 *>(sb + offsetof(RasterSetup, M)));
        const float4 m1 = __ldg(reinterpret_cast<const float4 *>(sb + offsetof(RasterSetup, M) + 16));
        const float4 m2 = __ldg(reinterpret_cast<const float4 *>(sb + offsetof(RasterSetup, M) + 32));
        const float4 t4 = __ldg(reinterpret_cast<const float4 *>(sb + offsetof(RasterSetup, t0)));
        const int4 bx = __ldg(reinterpret_cast<const int4 *>(sb + offsetof(RasterSetup, ilo)));
        const int2 bz2 = __ldg(reinterpret_cast<const int2 *>(sb + offsetof(RasterSetup, klo)));
        const DevProblem &P = probs[entries[e].prob];
        const int nx = P.nx, ny = P.ny;
        const int2 *brec = bandrows + (2 * (size_t)e + side) * kBandRows;
        const bool recorded = nband <= kBandRows;
        const int ilo = bx.x, ihi = bx.y, jlo = bx.z, klo = bz2.x;
        const int nyb = max(bx.w - jlo + 1, 1), nzb = bz2.y - klo + 1;
        const int n_rows = recorded ? nband : ((ilo <= ihi && bx.w >= jlo && nzb > 0) ? nyb * nzb : 0);
        float s_g = 0.0f, c_g = 0.0f;
        int dk = lane / nyb, dj = lane - dk * nyb;
        const int inc_k = 32 / nyb, inc_j = 32 - inc_k * nyb;
        for (int rb = 0; rb < n_rows; rb += 32) {
            int lo = 1, hi = 0, j = 0, k = 0;   // x range of the row part, then band-list positions
            if (recorded) {
                if (rb + lane < n_rows) {
                    const int2 rec = brec[rb + lane];
                    lo = rec.x & 0xffff;
                    hi = rec.x >> 16;
                    j = rec.y & 0xffff;
                    k = rec.y >> 16;
                }
            } else {
                j = jlo + dj;
                k = klo + dk;
                if (dk < nzb) {
                    row_interval(su->f, dj, dk, ilo, ihi, lo, hi);
                    if (hi >= lo) {
                        const short2 br = __ldg(P.bandrow[side] + (k * ny + j));
                        lo = max(lo, (int)br.x);
                        hi = min(hi, (int)br.y);
                    }
                }
                dj += inc_j;
                dk += inc_k;
                if (dj >= nyb) {
                    dj -= nyb;
                    dk += 1;
                }
            }
            // the band voxels of row (j, k) with lo <= x <= hi: positions [a, a + cnt)
            // of the row's list, from the per-voxel rank within the row
            int a = 0, cnt = 0;
            if (hi >= lo) {
                const int row = k * ny + j;
                const size_t rb = (size_t)row * nx;
                const int b0 = __ldg(P.band_start[side] + row);
                const int rlo = __ldg(P.band_rank[side] + rb + lo);
                const int rhi = __ldg(P.band_rank[side] + rb + hi);
                const int last = __ldg(P.band[side] + rb + hi) != 0 ? 1 : 0;
                a = b0 + rlo;
                cnt = rhi - rlo + last;
            }
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += v;
            }
            const int total = __shfl_sync(FULL, incl, 31);
            const int d = a - (incl - cnt);           // list position = d + v
            const int jk = j | (k << 16);
            // two 32-voxel chunks per pass: both chunks' records and samples are
            // loaded before either is summed; the lane sums voxel vb + lane, then
            // vb + 32 + lane, the order of one chunk per pass
            auto owner = [&](int v) {
                int ow = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const int p = __shfl_sync(FULL, incl, ow + step - 1);
                    if (p <= v) ow += step;
                }
                return ow;
            };
            for (int vb = 0; vb < total; vb += 64) {
                const int v0 = vb + lane, v1 = vb + 32 + lane;
                const int ow0 = owner(v0), ow1 = owner(v1);
                const int od0 = __shfl_sync(FULL, d, ow0), ojk0 = __shfl_sync(FULL, jk, ow0);
                const int od1 = __shfl_sync(FULL, d, ow1), ojk1 = __shfl_sync(FULL, jk, ow1);
                int2 r0 = make_int2(0, 0), r1 = make_int2(0, 0);
                if (v0 < total) r0 = __ldg(P.band_rec[side] + od0 + v0);
                if (v1 < total) r1 = __ldg(P.band_rec[side] + od1 + v1);
                BandVoxel b0, b1;
                if (v0 < total) b0 = band_load(P, side, m0, m1, m2, t4, r0, ojk0);
                if (v1 < total) b1 = band_load(P, side, m0, m1, m2, t4, r1, ojk1);
                if (v0 < total) band_sum(P, side, b0, s_g, c_g);
                if (v1 < total) band_sum(P, side, b1, s_g, c_g);
            }
        }
        const float e_g = warp_comp_sum(s_g, -c_g);
        if (lane == 0) {
            ro->e_guid = e_g;
            ro->n_gp = 0;
            const int pi = entries[e].prob;
            BatchClock *ck = P.clock;
            // batched evaluation: the image pass counted this problem's listed items before this kernel began
            if (ck && atomicAdd(&ck->guid_done[pi], 1) + 1 == ck->guid_total[pi]) ck->t_guid[pi] = global_ns();
        }
    });
}

template <typename TI, int HMODE, bool ORDERED>
cudaError_t launch_g(const DevProblem *probs, int g_mode, const WorkEntry *entries, const RasterSetup *setup,
                     RasterOut *rout, int2 *bandrows, const int *n_dev, int n_host, int grid, int chunk, int *queue,
                     const int *order, BatchClock *clock, cudaStream_t st)
{
    switch (g_mode) {
    case MOREA_G_CONTINUOUS:
        k_raster<TI, HMODE, kPassImageBand, ORDERED><<<grid, kBlock, 0, st>>>(probs, entries, setup, rout, bandrows,
                                                                             n_dev, n_host, chunk, queue, order, clock);
        if (cudaPeekAtLastError() == cudaSuccess)
            k_guidance<<<grid, kBlock, 0, st>>>(probs, entries, setup, rout, bandrows, n_dev, n_host, chunk,
                                                queue);
        break;
    case MOREA_G_PAIR_TRANSFER:
        k_raster<TI, HMODE, kPassImagePairs, ORDERED><<<grid, kBlock, 0, st>>>(probs, entries, setup, rout,
                                                                              bandrows, n_dev, n_host, chunk, queue,
                                                                              order, clock);
        break;
    default:
        k_raster<TI, HMODE, kPassImage, ORDERED><<<grid, kBlock, 0, st>>>(probs, entries, setup, rout, bandrows,
                                                                         n_dev, n_host, chunk, queue, order, clock);
        break;
    }
    return cudaGetLastError();
}

// Kernel variant of a launch: storage type, h mode and whether the items
// come in the entry pass's order.
template <typename TI, int HMODE>
cudaError_t launch_o(const DevProblem *probs, int g_mode, const WorkEntry *entries, const RasterSetup *setup,
                     RasterOut *rout, int2 *bandrows, const int *n_dev, int n_host, int grid, int chunk, int *queue,
                     const int *order, BatchClock *clock, cudaStream_t st)
{
    if (order)
        return launch_g<TI, HMODE, true>(probs, g_mode, entries, setup, rout, bandrows, n_dev, n_host, grid, chunk,
                                         queue, order, clock, st);
    return launch_g<TI, HMODE, false>(probs, g_mode, entries, setup, rout, bandrows, n_dev, n_host, grid, chunk,
                                      queue, nullptr, clock, st);
}

}  // namespace

cudaError_t launch_raster(const DevProblem *probs, const DevProblem &hp, const WorkEntry *entries,
                          const RasterSetup *setup, RasterOut *rout, int2 *bandrows, const int *n_entries_dev,
                          int n_entries_host, int grid, int chunk, int *queue, bool ordered, BatchClock *clock,
                          cudaStream_t st)
{
    const int *order = ordered ? queue + kQueueList + 2 * (size_t)n_entries_host : nullptr;
    if (grid <= 0) grid = sm_count() * 8;
    // the work counters and the guidance list; the large-item count of an
    // ordered pass was set by the entry pass and stays
    cudaError_t e = cudaMemsetAsync(queue, 0, kQueueOrderBig * sizeof(int), st);
    if (e != cudaSuccess) return e;

    if (hp.estimator == MOREA_EST_SAMPLED)
        return launch_sample(probs, hp, entries, setup, rout, n_entries_dev, n_entries_host, grid, chunk, queue, st);
    if (hp.dtype == MOREA_F16) {
        if (hp.h_mode == MOREA_H_MOREA_FG)
            return launch_o<__half, MOREA_H_MOREA_FG>(probs, hp.g_mode, entries, setup, rout, bandrows, n_entries_dev,
                                                      n_entries_host, grid, chunk, queue, order, clock, st);
        return launch_o<__half, MOREA_H_PLAIN_SSD>(probs, hp.g_mode, entries, setup, rout, bandrows, n_entries_dev,
                                                   n_entries_host, grid, chunk, queue, order, clock, st);
    }
    if (hp.h_mode == MOREA_H_MOREA_FG)
        return launch_o<float, MOREA_H_MOREA_FG>(probs, hp.g_mode, entries, setup, rout, bandrows, n_entries_dev,
                                                 n_entries_host, grid, chunk, queue, order, clock, st);
    return launch_o<float, MOREA_H_PLAIN_SSD>(probs, hp.g_mode, entries, setup, rout, bandrows, n_entries_dev,
                                              n_entries_host, grid, chunk, queue, order, clock, st);
}

}  // namespace morea
