// Device helpers shared by the image passes (k_raster.cu, k_sample.cu,
// k_dvf.cu): image and quad loads, trilinear sampling with the clamping of
// reading R4, h of Sec. 4.1.2, compensated FP32 accumulation and its warp
// reduction, the item scheduler, and the exact row intervals of a tet copy
// (reading R3).  Internal; each translation unit gets its own copy.
#pragma once

#include "morea_device.cuh"

namespace morea {

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <typename TI>
struct QuadOf;
template <>
struct QuadOf<float> {
    using T = float4;
};
template <>
struct QuadOf<__half> {
    using T = uint2;
};

__device__ __forceinline__ float ld_img(const float *p, int idx) { return __ldg(p + idx); }
__device__ __forceinline__ float ld_img(const __half *p, int idx) { return __half2float(__ldg(p + idx)); }

// one z-plane of the neighbourhood: (x,y), (x+1,y), (x,y+1), (x+1,y+1)
__device__ __forceinline__ void ld_quad(const float4 *q, int idx, float &a, float &b, float &c, float &d)
{
    const float4 v = __ldg(q + idx);
    a = v.x;
    b = v.y;
    c = v.z;
    d = v.w;
}

__device__ __forceinline__ void ld_quad(const uint2 *q, int idx, float &a, float &b, float &c, float &d)
{
    const uint2 v = __ldg(q + idx);
    const float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
    const float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
    a = lo.x;
    b = lo.y;
    c = hi.x;
    d = hi.y;
}

// Trilinear sample with the position clamped to [0, n-1] per axis and the
// cell i0 = min(floor(y), n - 2), from the quad copy of the image (q at the
// element of cell (0, 0, 0); row stride nx + 1, plane stride
// (nx + 1)(ny + 1)).
template <typename QT>
__device__ __forceinline__ float trilin_quad(const QT *q, int nx, int ny, int nz, float yx, float yy, float yz)
{
    const float cx = fminf(fmaxf(yx, 0.0f), (float)(nx - 1));
    const float cy = fminf(fmaxf(yy, 0.0f), (float)(ny - 1));
    const float cz = fminf(fmaxf(yz, 0.0f), (float)(nz - 1));
    const int ix = min((int)cx, nx - 2), iy = min((int)cy, ny - 2), iz = min((int)cz, nz - 2);
    const float fx = cx - (float)ix, fy = cy - (float)iy, fz = cz - (float)iz;
    const int sx = nx + 1, sxy = (nx + 1) * (ny + 1);
    const int b = iz * sxy + iy * sx + ix;
    float v000, v100, v010, v110, v001, v101, v011, v111;
    ld_quad(q, b, v000, v100, v010, v110);
    ld_quad(q, b + sxy, v001, v101, v011, v111);
    const float c00 = fmaf(fx, v100 - v000, v000), c10 = fmaf(fx, v110 - v010, v010);
    const float c01 = fmaf(fx, v101 - v001, v001), c11 = fmaf(fx, v111 - v011, v011);
    const float c0 = fmaf(fy, c10 - c00, c00), c1 = fmaf(fy, c11 - c01, c01);
    return fmaf(fz, c1 - c0, c0);
}

// The same sample when the position is known to lie in [-1, n) per axis:
// the padding of the quad copy repeats the edge values, so the cell
// floor(y) (from -1 to n - 1) gives the clamped sample without clamping:
// outside [0, n - 1] both corners of an axis hold the edge value, inside it
// the cell and weights are those of the clamped form.  sx = nx + 1,
// sxy = (nx + 1)(ny + 1).
template <typename QT>
__device__ __forceinline__ float trilin_quad_inner(const QT *q, int sx, int sxy, float yx, float yy, float yz)
{
    const int ix = __float2int_rd(yx), iy = __float2int_rd(yy), iz = __float2int_rd(yz);
    const float fx = yx - (float)ix, fy = yy - (float)iy, fz = yz - (float)iz;
    const int b = iz * sxy + iy * sx + ix;
    float v000, v100, v010, v110, v001, v101, v011, v111;
    ld_quad(q, b, v000, v100, v010, v110);
    ld_quad(q, b + sxy, v001, v101, v011, v111);
    const float c00 = fmaf(fx, v100 - v000, v000), c10 = fmaf(fx, v110 - v010, v010);
    const float c01 = fmaf(fx, v101 - v001, v001), c11 = fmaf(fx, v111 - v011, v011);
    const float c0 = fmaf(fy, c10 - c00, c00), c1 = fmaf(fy, c11 - c01, c01);
    return fmaf(fz, c1 - c0, c0);
}

// The same sample from a plain FP32 image (guidance distance maps).
__device__ __forceinline__ float trilin_plain(const float *img, int nx, int ny, int nz, float yx, float yy, float yz)
{
    const float cx = fminf(fmaxf(yx, 0.0f), (float)(nx - 1));
    const float cy = fminf(fmaxf(yy, 0.0f), (float)(ny - 1));
    const float cz = fminf(fmaxf(yz, 0.0f), (float)(nz - 1));
    const int ix = min((int)cx, nx - 2), iy = min((int)cy, ny - 2), iz = min((int)cz, nz - 2);
    const float fx = cx - (float)ix, fy = cy - (float)iy, fz = cz - (float)iz;
    const int sy = nx, sz = nx * ny;
    const int b = (iz * ny + iy) * nx + ix;
    const float v000 = __ldg(img + b), v100 = __ldg(img + b + 1);
    const float v010 = __ldg(img + b + sy), v110 = __ldg(img + b + sy + 1);
    const float v001 = __ldg(img + b + sz), v101 = __ldg(img + b + sz + 1);
    const float v011 = __ldg(img + b + sz + sy), v111 = __ldg(img + b + sz + sy + 1);
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

// Item scheduling of the image and guidance passes: static striding of the
// (entry, side) items over all warps, or (chunk > 0) a work queue from which
// each warp takes `chunk` consecutive items with one atomic add, so warps that
// drew large tets do not hold up the tail of an uneven batch.
template <typename F>
__device__ __forceinline__ void run_items(int n_items, int chunk, int *queue, F &&body)
{
    const int lane = threadIdx.x & 31;
    if (chunk <= 0) {
        const int wpb = blockDim.x >> 5;
        for (int item = blockIdx.x * wpb + (threadIdx.x >> 5); item < n_items; item += gridDim.x * wpb) body(item);
        return;
    }
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(queue, chunk);
        base = __shfl_sync(FULL, base, 0);
        if (base >= n_items) break;
        const int end = min(base + chunk, n_items);
        for (int item = base; item < end; ++item) body(item);
    }
}

// ---- exact voxel association of one tet copy (reading R3) ----

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

// Exact x-interval [lo, hi] of the voxel centres of row (jlo + dj, klo + dk).
// Per face the FP32 root estimate decides whenever it is farther than the
// face's error bound from the bounding-box ends and from every integer;
// otherwise the bound is solved exactly in int64.
// Loads of a copy's face rows: through the read-only data cache when the
// rows are in global memory (the image passes), plain loads when a caller
// keeps them in shared memory (k_dvf); ld.global.nc must never see a shared
// address.
template <bool GLOBAL, typename T>
__device__ __forceinline__ T face_load(const T *p)
{
    if (GLOBAL) return __ldg(p);
    return *p;
}

template <bool GLOBAL = true>
__device__ __forceinline__ void row_interval(const FaceRow *__restrict__ f, int dj, int dk, int ilo, int ihi,
                                             int &lo, int &hi)
{
    lo = ilo;
    hi = ihi;
    const float fdj = (float)dj, fdk = (float)dk;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 es = face_load<GLOBAL>(reinterpret_cast<const float4 *>(&f[q].e0));       // e0, ey, ez, signed tol
        if (isinf(es.w)) {                    // face parallel to x: the whole row or nothing
            const longlong2 ab = face_load<GLOBAL>(reinterpret_cast<const longlong2 *>(&f[q].ax));
            const longlong2 yz = face_load<GLOBAL>(reinterpret_cast<const longlong2 *>(&f[q].by));
            if (ab.y + yz.x * dj + yz.y * dk <= 0) hi = lo - 1;
            continue;
        }
        const float est = fmaf(es.y, fdj, fmaf(es.z, fdk, es.x));
        const float tol = fabsf(es.w);
        const float fl = floorf(est);
        const float fr = est - fl;
        if (es.w > 0.0f) {                    // ax > 0, inside for i > root: lo = floor(root) + 1
            if (est + tol < (float)ilo) continue;
            if (est - tol >= (float)ihi) { hi = lo - 1; continue; }
            if (fr > tol && fr < 1.0f - tol) { lo = max(lo, (int)fl + 1); continue; }
            const longlong2 ab = face_load<GLOBAL>(reinterpret_cast<const longlong2 *>(&f[q].ax));
            const longlong2 yz = face_load<GLOBAL>(reinterpret_cast<const longlong2 *>(&f[q].by));
            lo = max(lo, face_lo(ab.x, ab.y + yz.x * dj + yz.y * dk, est, ilo, ihi));
        } else {                              // ax < 0, inside for i < root: hi = ceil(root) - 1
            if (est - tol > (float)ihi) continue;
            if (est + tol <= (float)ilo) { hi = lo - 1; continue; }
            if (fr > tol && fr < 1.0f - tol) { hi = min(hi, (int)fl); continue; }
            const longlong2 ab = face_load<GLOBAL>(reinterpret_cast<const longlong2 *>(&f[q].ax));
            const longlong2 yz = face_load<GLOBAL>(reinterpret_cast<const longlong2 *>(&f[q].by));
            hi = min(hi, face_hi(ab.x, ab.y + yz.x * dj + yz.y * dk, est, ilo, ihi));
        }
    }
}

// y-extent [y0, y1] (snapped units) of the cross-section of a tet copy with
// the plane z = zq: the intersections of its six edges with the plane.  The
// vertices are integers below 2^17, so each intersection is within 2^-6 of
// its exact value (one rounded division and one FMA); callers widen the
// extent by more than that.  Empty (y0 > y1) if no edge meets the plane.
__device__ __forceinline__ void slice_y_extent(const int4 *vq, float zq, float &y0, float &y1)
{
    float y[4], z[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int4 t = __ldg(vq + v);
        y[v] = (float)t.y;
        z[v] = (float)t.z;
    }
    y0 = INFINITY;
    y1 = -INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a + 1; b < 4; ++b) {
            if (fminf(z[a], z[b]) <= zq && zq <= fmaxf(z[a], z[b])) {
                float ya = y[a], yb = y[b];
                if (z[a] != z[b]) ya = yb = fmaf((zq - z[a]) / (z[b] - z[a]), y[b] - y[a], y[a]);
                y0 = fminf(y0, fminf(ya, yb));
                y1 = fmaxf(y1, fmaxf(ya, yb));
            }
        }
}

}  // namespace

}  // namespace morea
