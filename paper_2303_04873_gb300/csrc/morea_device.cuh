// Device helpers shared by the kernels of libmorea (snap, exact orientation,
// per-tet set-up, fold and magnitude terms).
#pragma once

#include "morea_internal.cuh"

namespace morea {

// Clamp to the image box and snap onto the 2^-k grid, round half to even:
// q = rint((x + 1/2) 2^k) = rint(x 2^k) + 2^(k-1) for k >= 2 (the shift is
// even, so it commutes with round-half-even).  x 2^k is exact in FP32.
__device__ __forceinline__ int snap1(float x, int n, int kbits, int H)
{
    float c = fminf(fmaxf(x, -0.5f), (float)n - 0.5f);
    return __float2int_rn(c * (float)(1 << kbits)) + H;
}

__device__ __forceinline__ int4 snap3(const float *p, const DevProblem &P)
{
    return make_int4(snap1(p[0], P.nx, P.kbits, P.H), snap1(p[1], P.ny, P.kbits, P.H),
                     snap1(p[2], P.nz, P.kbits, P.H), 0);
}

// orient(a,b,c,d) = (b-a).((c-a)x(d-a)), six times the signed volume.  With
// coordinates in [0, 2^16] every product and partial sum is an integer below
// 2^53, so FP64 evaluates it exactly in any order (Sec. 4.1.4 / App. A.4).
__device__ __forceinline__ double orient_d(int4 a, int4 b, int4 c, int4 d)
{
    double bx = b.x - a.x, by = b.y - a.y, bz = b.z - a.z;
    double cx = c.x - a.x, cy = c.y - a.y, cz = c.z - a.z;
    double dx = d.x - a.x, dy = d.y - a.y, dz = d.z - a.z;
    return bx * (cy * dz - cz * dy) + by * (cz * dx - cx * dz) + bz * (cx * dy - cy * dx);
}

__device__ __forceinline__ int floor_shift(int a, int k) { return a >> k; }        // floor(a / 2^k)
__device__ __forceinline__ int ceil_shift(int a, int k) { return -((-a) >> k); }   // ceil(a / 2^k)

// (|e_s| - |e_t|)^2 * scale^2 with the difference formed from the exact
// integer squared lengths: (l2s - l2t) / (sqrt(l2s) + sqrt(l2t)); no
// cancellation when the two lengths are close.
__device__ __forceinline__ float len_diff_sq(long long l2s, long long l2t, float scale)
{
    long long d = l2s - l2t;
    if (d == 0) return 0.0f;
    float den = sqrtf((float)l2s) + sqrtf((float)l2t);
    float diff = (float)d / den * scale;
    return diff * diff;
}

__device__ __forceinline__ long long sq3(long long x, long long y, long long z) { return x * x + y * y + z * z; }

// Deformation magnitude of one tet (Sec. 4.1.1): 6 edges + 4 centroid
// spokes, c_delta * sum (|e_s| - |e_t|)^2 in voxel units.  Fold flags and
// the integer severity of the two copies (App. A.4).
__device__ __forceinline__ void tet_terms(const int4 *qs, const int4 *qt, const DevProblem &P, int t,
                                          TetOut &o)
{
    double Ds = orient_d(qs[0], qs[1], qs[2], qs[3]);
    double Dt = orient_d(qt[0], qt[1], qt[2], qt[3]);
    unsigned int folded = 0;
    unsigned long long sev = 0;
    if (Ds <= 0.0) { folded |= 1u; sev += (unsigned long long)(-Ds); }
    if (Dt <= 0.0) { folded |= 2u; sev += (unsigned long long)(-Dt); }
    const float inv_s = 1.0f / (float)P.S;
    float e = 0.0f;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a + 1; b < 4; ++b) {
            long long ls = sq3(qs[b].x - qs[a].x, qs[b].y - qs[a].y, qs[b].z - qs[a].z);
            long long lt = sq3(qt[b].x - qt[a].x, qt[b].y - qt[a].y, qt[b].z - qt[a].z);
            e += len_diff_sq(ls, lt, inv_s);
        }
    const int csx = qs[0].x + qs[1].x + qs[2].x + qs[3].x, csy = qs[0].y + qs[1].y + qs[2].y + qs[3].y,
              csz = qs[0].z + qs[1].z + qs[2].z + qs[3].z;
    const int ctx = qt[0].x + qt[1].x + qt[2].x + qt[3].x, cty = qt[0].y + qt[1].y + qt[2].y + qt[3].y,
              ctz = qt[0].z + qt[1].z + qt[2].z + qt[3].z;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        // spoke vector in units of 2^-k / 4: 4 v_a - sum v
        long long ls = sq3(4LL * qs[a].x - csx, 4LL * qs[a].y - csy, 4LL * qs[a].z - csz);
        long long lt = sq3(4LL * qt[a].x - ctx, 4LL * qt[a].y - cty, 4LL * qt[a].z - ctz);
        e += len_diff_sq(ls, lt, 0.25f * inv_s);
    }
    o.e_mag = P.cdelta[t] * e;
    o.folded = folded;
    o.sev = sev;
}

// Rasterisation set-up of one tet copy ("own") against the other copy.
// D_f(p) = orientation with vertex f replaced by p = (-1)^(f+1) N_f.(p - w0),
// N_f = (w1 - w0) x (w2 - w0) over the other three vertices in order.
__device__ __forceinline__ void make_setup(const int4 *own, const int4 *oth, const DevProblem &P,
                                           RasterSetup &su)
{
    const double D = orient_d(own[0], own[1], own[2], own[3]);
    const int kb = P.kbits, H = P.H;
    int mnx = min(min(own[0].x, own[1].x), min(own[2].x, own[3].x));
    int mxx = max(max(own[0].x, own[1].x), max(own[2].x, own[3].x));
    int mny = min(min(own[0].y, own[1].y), min(own[2].y, own[3].y));
    int mxy = max(max(own[0].y, own[1].y), max(own[2].y, own[3].y));
    int mnz = min(min(own[0].z, own[1].z), min(own[2].z, own[3].z));
    int mxz = max(max(own[0].z, own[1].z), max(own[2].z, own[3].z));
    su.ilo = max(0, ceil_shift(mnx - H, kb));
    su.ihi = min(P.nx - 1, floor_shift(mxx - H, kb));
    su.jlo = max(0, ceil_shift(mny - H, kb));
    su.jhi = min(P.ny - 1, floor_shift(mxy - H, kb));
    su.klo = max(0, ceil_shift(mnz - H, kb));
    su.khi = min(P.nz - 1, floor_shift(mxz - H, kb));
    su.qlo[0] = mnx; su.qlo[1] = mny; su.qlo[2] = mnz;
    su.qhi[0] = mxx; su.qhi[1] = mxy; su.qhi[2] = mxz;
    // the other copy's bounding box strictly inside (-1, n) (margin 1/64
    // voxel, far above the FP32 error of a mapped position): then the
    // trilinear sample from the padded quad copy needs no clamping (every
    // snapped point lies in [-0.5, n - 0.5], so this holds for every copy)
    bool inner = true;
    {
        const int om[3] = {min(min(oth[0].x, oth[1].x), min(oth[2].x, oth[3].x)),
                           min(min(oth[0].y, oth[1].y), min(oth[2].y, oth[3].y)),
                           min(min(oth[0].z, oth[1].z), min(oth[2].z, oth[3].z))};
        const int oM[3] = {max(max(oth[0].x, oth[1].x), max(oth[2].x, oth[3].x)),
                           max(max(oth[0].y, oth[1].y), max(oth[2].y, oth[3].y)),
                           max(max(oth[0].z, oth[1].z), max(oth[2].z, oth[3].z))};
        const int n[3] = {P.nx, P.ny, P.nz};
        const int margin = max(1, P.S >> 6);
        for (int a = 0; a < 3; ++a)
            inner = inner && om[a] - H >= margin - P.S && oM[a] - H <= n[a] * P.S - margin;
    }
    su.valid = (D > 0.0 ? 1 : 0) | (inner ? 2 : 0);
    const long long S = P.S;
    const int nyb1 = max(0, su.jhi - su.jlo), nzb1 = max(0, su.khi - su.klo);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        int4 w0 = own[f == 0 ? 1 : 0];
        int4 w1 = own[f <= 1 ? 2 : 1];
        int4 w2 = own[f <= 2 ? 3 : 2];
        long long ux = w1.x - w0.x, uy = w1.y - w0.y, uz = w1.z - w0.z;
        long long vx = w2.x - w0.x, vy = w2.y - w0.y, vz = w2.z - w0.z;
        long long nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
        if ((f & 1) == 0) { nx = -nx; ny = -ny; nz = -nz; }
        long long c = -(nx * w0.x + ny * w0.y + nz * w0.z);
        // simulation of simplicity: a zero value takes the sign of the first
        // nonzero gradient component (x, then y, then z)
        long long tie = (nx > 0 || (nx == 0 && (ny > 0 || (ny == 0 && nz > 0)))) ? 1 : 0;
        long long ct = c + tie;
        su.ct[f] = ct;
        FaceRow fr;
        fr.ax = nx * S;
        fr.by = ny * S;
        fr.bz = nz * S;
        fr.b00 = ct + (nx + ny + nz) * (long long)H + fr.by * su.jlo + fr.bz * su.klo;
        if (nx != 0) {
            double inv = -1.0 / (double)fr.ax;
            fr.e0 = (float)((double)fr.b00 * inv);
            fr.ey = (float)((double)fr.by * inv);
            fr.ez = (float)((double)fr.bz * inv);
            // |estimate - root| <= 2^-24 (3 |e0| + 3 |ey| dj + 3 |ez| dk) (rounding
            // of e0, ey, ez and of the two FMAs); 2^-20 leaves a factor 5 margin
            // stored with the sign of ax, so the row test needs no int64 load
            // to know on which side of the root the inside lies
            const float tol = (fabsf(fr.e0) + fabsf(fr.ey) * (float)nyb1 + fabsf(fr.ez) * (float)nzb1 + 1.0f) *
                              (1.0f / 1048576.0f);
            fr.tol = nx > 0 ? tol : -tol;
        } else {
            fr.e0 = fr.ey = fr.ez = 0.0f;
            fr.tol = INFINITY;                // face parallel to x: exact test of the whole row
        }
        su.f[f] = fr;
    }
    // affine map own -> other: M = F E^-1, E = [e1 e2 e3] edge columns of the
    // own copy, rows of E^-1 = (e2 x e3, e3 x e1, e1 x e2) / D (exact int64
    // numerators, one FP64 division each).
    long long e1x = own[1].x - own[0].x, e1y = own[1].y - own[0].y, e1z = own[1].z - own[0].z;
    long long e2x = own[2].x - own[0].x, e2y = own[2].y - own[0].y, e2z = own[2].z - own[0].z;
    long long e3x = own[3].x - own[0].x, e3y = own[3].y - own[0].y, e3z = own[3].z - own[0].z;
    long long r1[3] = {e2y * e3z - e2z * e3y, e2z * e3x - e2x * e3z, e2x * e3y - e2y * e3x};
    long long r2[3] = {e3y * e1z - e3z * e1y, e3z * e1x - e3x * e1z, e3x * e1y - e3y * e1x};
    long long r3[3] = {e1y * e2z - e1z * e2y, e1z * e2x - e1x * e2z, e1x * e2y - e1y * e2x};
    long long f1[3] = {oth[1].x - oth[0].x, oth[1].y - oth[0].y, oth[1].z - oth[0].z};
    long long f2[3] = {oth[2].x - oth[0].x, oth[2].y - oth[0].y, oth[2].z - oth[0].z};
    long long f3[3] = {oth[3].x - oth[0].x, oth[3].y - oth[0].y, oth[3].z - oth[0].z};
    const double invD = D > 0.0 ? 1.0 / D : 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            su.M[3 * a + b] = (float)((double)(f1[a] * r1[b] + f2[a] * r2[b] + f3[a] * r3[b]) * invD);
    const float inv_s = 1.0f / (float)P.S;
    su.s0[0] = own[0].x * inv_s - 0.5f;
    su.s0[1] = own[0].y * inv_s - 0.5f;
    su.s0[2] = own[0].z * inv_s - 0.5f;
    su.t0[0] = oth[0].x * inv_s - 0.5f;
    su.t0[1] = oth[0].y * inv_s - 0.5f;
    su.t0[2] = oth[0].z * inv_s - 0.5f;
}

// A large item of the image pass: an unfolded copy whose bounding box holds
// at least kBigItemVoxels voxel centres.
__device__ __forceinline__ bool item_is_big(const RasterSetup &su)
{
    return (su.valid & 1) && (long long)max(su.ihi - su.ilo + 1, 0) * max(su.jhi - su.jlo + 1, 0) *
                                     max(su.khi - su.klo + 1, 0) >= kBigItemVoxels;
}

}  // namespace morea
