// The hot loop of libmorea (steps a4-a7): for each (work entry, side) one
// warp walks the voxel-centre rows of the tet copy's bounding box, solves the
// exact integer x-interval of each row, spreads the row's voxels over the
// 32 lanes, maps every voxel centre p into the other image with the tet's
// affine map, samples the other image trilinearly, accumulates h (Sec. 4.1.2)
// and the continuous guidance term (Sec. 4.1.3) in compensated FP32, and
// reduces the per-lane sums with warp shuffles into one record per
// (entry, side).
//
// Voxel association (exact): a voxel centre P is inside the copy iff for
// every face f: A_f i + B_f(j, k) > 0 (integers, simulation-of-simplicity tie
// bit folded into B).  Each face bound is first estimated in FP32 and then
// corrected with exact int64 evaluations, so the interval does not depend on
// the estimate's rounding.
#include "morea_device.cuh"

namespace morea {

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <typename TI>
__device__ __forceinline__ float ld_img(const TI *p, int idx);

template <>
__device__ __forceinline__ float ld_img<float>(const float *p, int idx)
{
    return __ldg(p + idx);
}

template <>
__device__ __forceinline__ float ld_img<__half>(const __half *p, int idx)
{
    return __half2float(__ldg(p + idx));
}

// Trilinear sample with the position clamped to [0, n-1] per axis and the
// cell i0 = min(floor(y), n - 2).
template <typename TI>
__device__ __forceinline__ float trilin(const TI *img, int nx, int ny, int nz, float yx, float yy, float yz)
{
    const float cx = fminf(fmaxf(yx, 0.0f), (float)(nx - 1));
    const float cy = fminf(fmaxf(yy, 0.0f), (float)(ny - 1));
    const float cz = fminf(fmaxf(yz, 0.0f), (float)(nz - 1));
    const int ix = min((int)cx, nx - 2), iy = min((int)cy, ny - 2), iz = min((int)cz, nz - 2);
    const float fx = cx - (float)ix, fy = cy - (float)iy, fz = cz - (float)iz;
    const int sy = nx, sz = nx * ny;
    const int b = (iz * ny + iy) * nx + ix;
    const float v000 = ld_img(img, b), v100 = ld_img(img, b + 1);
    const float v010 = ld_img(img, b + sy), v110 = ld_img(img, b + sy + 1);
    const float v001 = ld_img(img, b + sz), v101 = ld_img(img, b + sz + 1);
    const float v011 = ld_img(img, b + sz + sy), v111 = ld_img(img, b + sz + sy + 1);
    const float c00 = fmaf(fx, v100 - v000, v000), c10 = fmaf(fx, v110 - v010, v010);
    const float c01 = fmaf(fx, v101 - v001, v001), c11 = fmaf(fx, v111 - v011, v011);
    const float c0 = fmaf(fy, c10 - c00, c00), c1 = fmaf(fy, c11 - c01, c01);
    return fmaf(fz, c1 - c0, c0);
}

template <int HMODE>
__device__ __forceinline__ float hfun(float a, float b)
{
    const float d = a - b;
    if (HMODE == MOREA_H_PLAIN_SSD) return d * d;
    if (a > 0.0f && b > 0.0f) return d * d;
    if (a == 0.0f && b == 0.0f) return 0.0f;
    return 1.0f;
}

// Kahan-compensated accumulation; (s, c) holds s - c.
__device__ __forceinline__ void kadd(float &s, float &c, float x)
{
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// Warp reduction of compensated pairs (hi, lo): error-free two-sum of the
// high parts, low parts and errors summed separately.
__device__ __forceinline__ float warp_comp_sum(float hi, float lo)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(FULL, hi, o);
        const float l2 = __shfl_xor_sync(FULL, lo, o);
        const float s = __fadd_rn(hi, h2);
        const float bp = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(h2, bp));
        hi = s;
        lo = __fadd_rn(__fadd_rn(lo, l2), err);
    }
    return __fadd_rn(hi, lo);
}

// Smallest i in [ilo, ihi + 1] with A i + B > 0 (A > 0); ihi + 1 if none.
__device__ __forceinline__ int face_lo(long long A, long long B, float est, int ilo, int ihi)
{
    const float ec = fminf(fmaxf(est, (float)(ilo - 1)), (float)(ihi + 1));
    int i = (int)floorf(ec) + 1;
    i = min(max(i, ilo), ihi + 1);
    while (i > ilo && A * (long long)(i - 1) + B > 0) --i;
    while (i <= ihi && A * (long long)i + B <= 0) ++i;
    return i;
}

// Largest i in [ilo - 1, ihi] with A i + B > 0 (A < 0); ilo - 1 if none.
__device__ __forceinline__ int face_hi(long long A, long long B, float est, int ilo, int ihi)
{
    const float ec = fminf(fmaxf(est, (float)(ilo - 1)), (float)(ihi + 1));
    int i = (int)ceilf(ec) - 1;
    i = min(max(i, ilo - 1), ihi);
    while (i < ihi && A * (long long)(i + 1) + B > 0) ++i;
    while (i >= ilo && A * (long long)i + B <= 0) --i;
    return i;
}

template <typename TI, int HMODE, int GMODE>
__global__ void __launch_bounds__(kBlock) k_raster(const DevProblem *__restrict__ probs,
                                                  const WorkEntry *__restrict__ entries,
                                                  const RasterSetup *__restrict__ setup,
                                                  RasterOut *__restrict__ rout, const int *n_entries_dev,
                                                  int n_entries_host)
{
    const int lane = threadIdx.x & 31;
    const int n_ent = n_entries_dev ? min(*n_entries_dev, n_entries_host) : n_entries_host;
    const int n_items = 2 * n_ent;
    const int wpb = blockDim.x >> 5;
    const int nwarps = gridDim.x * wpb;
    for (int item = blockIdx.x * wpb + (threadIdx.x >> 5); item < n_items; item += nwarps) {
        const int side = item >= n_ent ? 1 : 0;      // all source sides first, then all target sides
        const int e = item - side * n_ent;
        const RasterSetup *su = setup + 2 * (size_t)e + side;
        float s_img = 0.0f, c_img = 0.0f, s_g = 0.0f, c_g = 0.0f;
        int nvox = 0, ngp = 0;
        if (su->valid) {
            const DevProblem &P = probs[entries[e].prob];
            const int nx = P.nx, ny = P.ny, nz = P.nz;
            const TI *own = (const TI *)P.img[side];
            const TI *oth = (const TI *)P.img[1 - side];
            const int ilo = su->ilo, ihi = su->ihi, jlo = su->jlo, klo = su->klo;
            const int nyb = su->jhi - jlo + 1, nzb = su->khi - klo + 1;
            const int n_rows = (ilo <= ihi && nyb > 0 && nzb > 0) ? nyb * nzb : 0;
            const float M0 = su->M[0], M1 = su->M[1], M2 = su->M[2];
            const float M3 = su->M[3], M4 = su->M[4], M5 = su->M[5];
            const float M6 = su->M[6], M7 = su->M[7], M8 = su->M[8];
            const float s0x = su->s0[0], s0y = su->s0[1], s0z = su->s0[2];
            const float t0x = su->t0[0], t0y = su->t0[1], t0z = su->t0[2];
            for (int rb = 0; rb < n_rows; rb += 32) {
                const int r = rb + lane;
                int lo = 1, hi = 0, j = 0, k = 0;
                if (r < n_rows) {
                    const int dk = r / nyb, dj = r - dk * nyb;
                    j = jlo + dj;
                    k = klo + dk;
                    lo = ilo;
                    hi = ihi;
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        const long long A = su->ax[f];
                        const long long B = su->b00[f] + su->by[f] * dj + su->bz[f] * dk;
                        if (A > 0) {
                            const float est = fmaf(su->ey[f], (float)dj, fmaf(su->ez[f], (float)dk, su->e0[f]));
                            lo = max(lo, face_lo(A, B, est, ilo, ihi));
                        } else if (A < 0) {
                            const float est = fmaf(su->ey[f], (float)dj, fmaf(su->ez[f], (float)dk, su->e0[f]));
                            hi = min(hi, face_hi(A, B, est, ilo, ihi));
                        } else if (B <= 0) {
                            lo = 1;
                            hi = 0;
                        }
                    }
                }
                const int cnt = max(0, hi - lo + 1);
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += v;
                }
                const int total = __shfl_sync(FULL, incl, 31);
                nvox += total;
                const int excl = incl - cnt;
                for (int vb = 0; vb < total; vb += 32) {
                    const int v = vb + lane;
                    int own_l = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        const int p = __shfl_sync(FULL, incl, own_l + step - 1);
                        if (p <= v) own_l += step;
                    }
                    const int ox = __shfl_sync(FULL, lo, own_l);
                    const int oe = __shfl_sync(FULL, excl, own_l);
                    const int oj = __shfl_sync(FULL, j, own_l);
                    const int ok = __shfl_sync(FULL, k, own_l);
                    if (v < total) {
                        const int x = ox + (v - oe);
                        const int idx = (ok * ny + oj) * nx + x;
                        const float a = ld_img(own, idx);
                        const float dx = (float)x - s0x, dy = (float)oj - s0y, dz = (float)ok - s0z;
                        const float yx = fmaf(M0, dx, fmaf(M1, dy, fmaf(M2, dz, t0x)));
                        const float yy = fmaf(M3, dx, fmaf(M4, dy, fmaf(M5, dz, t0y)));
                        const float yz = fmaf(M6, dx, fmaf(M7, dy, fmaf(M8, dz, t0z)));
                        const float b = trilin(oth, nx, ny, nz, yx, yy, yz);
                        kadd(s_img, c_img, hfun<HMODE>(a, b));
                        if (GMODE == MOREA_G_CONTINUOUS) {
                            unsigned mk = P.band[side][idx];
                            while (mk) {
                                const int g = __ffs(mk) - 1;
                                mk &= mk - 1;
                                const size_t off = (size_t)g * ((size_t)nx * ny * nz);
                                const float av = __ldg(P.dmap[side] + off + idx);
                                if (av < P.r) {
                                    const float dv = trilin(P.dmap[1 - side] + off, nx, ny, nz, yx, yy, yz);
                                    const float w = P.wgt[g] * (P.r - av) * P.inv_r;
                                    const float df = av - dv;
                                    kadd(s_g, c_g, w * df * df);
                                }
                            }
                        }
                    }
                }
            }
            if (GMODE == MOREA_G_PAIR_TRANSFER && P.n_guid > 0) {
                // guidance points of this side located in the copy (exact
                // perturbed inside test on their snapped coordinates)
                const int cs = P.cshift;
                const int cx0 = max(0, su->qlo[0] >> cs), cx1 = min(P.cgx - 1, su->qhi[0] >> cs);
                const int cy0 = max(0, su->qlo[1] >> cs), cy1 = min(P.cgy - 1, su->qhi[1] >> cs);
                const int cz0 = max(0, su->qlo[2] >> cs), cz1 = min(P.cgz - 1, su->qhi[2] >> cs);
                const int kb = P.kbits;
                const float inv_s = 1.0f / (float)P.S;
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
                                    const long long val = (su->ax[f] >> kb) * q.x + (su->by[f] >> kb) * q.y +
                                                          (su->bz[f] >> kb) * q.z + su->ct[f];
                                    in = in && val > 0;
                                }
                                if (in) {
                                    const float dx = q.x * inv_s - 0.5f - s0x;
                                    const float dy = q.y * inv_s - 0.5f - s0y;
                                    const float dz = q.z * inv_s - 0.5f - s0z;
                                    const float4 go = P.gp[1 - side][mi];
                                    const float ex = fmaf(M0, dx, fmaf(M1, dy, fmaf(M2, dz, t0x))) - go.x;
                                    const float ey = fmaf(M3, dx, fmaf(M4, dy, fmaf(M5, dz, t0y))) - go.y;
                                    const float ez = fmaf(M6, dx, fmaf(M7, dy, fmaf(M8, dz, t0z))) - go.z;
                                    kadd(s_g, c_g, fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
                                    ngp += 1;
                                }
                            }
                        }
            }
        }
        const float e_img = warp_comp_sum(s_img, -c_img);
        const float e_g = warp_comp_sum(s_g, -c_g);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ngp += __shfl_xor_sync(FULL, ngp, o);
        if (lane == 0) {
            RasterOut ro;
            ro.e_img = e_img;
            ro.e_guid = e_g;
            ro.n_vox = nvox;
            ro.n_gp = ngp;
            rout[2 * (size_t)e + side] = ro;
        }
    }
}

template <typename TI, int HMODE>
cudaError_t launch_g(const DevProblem *probs, int g_mode, const WorkEntry *entries, const RasterSetup *setup,
                     RasterOut *rout, const int *n_dev, int n_host, int grid, cudaStream_t st)
{
    switch (g_mode) {
    case MOREA_G_CONTINUOUS:
        k_raster<TI, HMODE, MOREA_G_CONTINUOUS><<<grid, kBlock, 0, st>>>(probs, entries, setup, rout, n_dev, n_host);
        break;
    case MOREA_G_PAIR_TRANSFER:
        k_raster<TI, HMODE, MOREA_G_PAIR_TRANSFER><<<grid, kBlock, 0, st>>>(probs, entries, setup, rout, n_dev,
                                                                           n_host);
        break;
    default:
        k_raster<TI, HMODE, MOREA_G_OFF><<<grid, kBlock, 0, st>>>(probs, entries, setup, rout, n_dev, n_host);
        break;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_raster(const DevProblem *probs, const DevProblem &hp, const WorkEntry *entries,
                          const RasterSetup *setup, RasterOut *rout, const int *n_entries_dev,
                          int n_entries_host, int grid, cudaStream_t st)
{
    if (grid <= 0) grid = sm_count() * 8;
    if (hp.dtype == MOREA_F16) {
        if (hp.h_mode == MOREA_H_MOREA_FG)
            return launch_g<__half, MOREA_H_MOREA_FG>(probs, hp.g_mode, entries, setup, rout, n_entries_dev,
                                                      n_entries_host, grid, st);
        return launch_g<__half, MOREA_H_PLAIN_SSD>(probs, hp.g_mode, entries, setup, rout, n_entries_dev,
                                                   n_entries_host, grid, st);
    }
    if (hp.h_mode == MOREA_H_MOREA_FG)
        return launch_g<float, MOREA_H_MOREA_FG>(probs, hp.g_mode, entries, setup, rout, n_entries_dev,
                                                 n_entries_host, grid, st);
    return launch_g<float, MOREA_H_PLAIN_SSD>(probs, hp.g_mode, entries, setup, rout, n_entries_dev,
                                              n_entries_host, grid, st);
}

}  // namespace morea
