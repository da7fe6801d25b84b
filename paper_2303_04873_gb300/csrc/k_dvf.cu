// Displacement field of one solution and the label overlap it implies (the
// evaluation of Sec. 5): for every voxel centre p of one image inside an
// unfolded copy (exact association, reading R3), dvf(p) = T(p) - p with the
// copy's FP32 affine map, and the label of the other image at the voxel
// nearest to T(p) (round half to even, clamped), counted against the own
// label and/or written out as the warped label image.
//
// One warp per tet: lane 0 builds the copy's rasterisation set-up in shared
// memory, the lanes take the rows of its bounding box and walk their
// voxels.  Voxels in no copy keep the NaN the field is filled with; with
// exact association and an unfolded conforming mesh each voxel is written
// once.  Per-label counts are gathered in a shared histogram per block and
// added to the output with 64-bit atomics.
#include "image_ops.cuh"

namespace morea {

namespace {

constexpr int kDvfWarps = 8;
constexpr int kMaxLabels = 64;

__global__ void __launch_bounds__(kDvfWarps * 32) k_dvf(const DevProblem *__restrict__ dp, const float *__restrict__ src,
                                                        const float *__restrict__ tgt, int side, float *__restrict__ dvf,
                                                        const uint8_t *__restrict__ lab_own,
                                                        const uint8_t *__restrict__ lab_oth, int n_labels,
                                                        unsigned long long *__restrict__ counts,
                                                        uint8_t *__restrict__ warped)
{
    __shared__ RasterSetup sus[kDvfWarps];
    __shared__ unsigned long long hist[kMaxLabels][3];
    const DevProblem &P = *dp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool labels = counts != nullptr, pull = labels || warped != nullptr;
    for (int i = threadIdx.x; i < kMaxLabels * 3; i += blockDim.x) (&hist[0][0])[i] = 0ull;
    __syncthreads();
    RasterSetup &su = sus[warp];
    const float *Xo = side == 0 ? src : tgt, *Xt = side == 0 ? tgt : src;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    for (int t = blockIdx.x * kDvfWarps + warp; t < P.n_tets; t += gridDim.x * kDvfWarps) {
        if (lane == 0) {
            const int4 tv = P.tets[t];
            const int ids[4] = {tv.x, tv.y, tv.z, tv.w};
            int4 own[4], oth[4];
            for (int i = 0; i < 4; ++i) {
                own[i] = snap3(Xo + 3 * (size_t)ids[i], P);
                oth[i] = snap3(Xt + 3 * (size_t)ids[i], P);
            }
            make_setup(own, oth, P, su);
        }
        __syncwarp();
        if (su.valid & 1) {
            const int ilo = su.ilo, ihi = su.ihi, jlo = su.jlo, klo = su.klo;
            const int nyb = su.jhi - jlo + 1, nzb = su.khi - klo + 1;
            const int n_rows = (ilo <= ihi && nyb > 0 && nzb > 0) ? nyb * nzb : 0;
            const float *M = su.M;
            for (int r = lane; r < n_rows; r += 32) {
                const int dk = r / nyb, dj = r - dk * nyb;
                int lo, hi;
                row_interval<false>(su.f, dj, dk, ilo, ihi, lo, hi);   // set-up in shared memory
                const int j = jlo + dj, k = klo + dk;
                const float dy = (float)j - su.s0[1], dz = (float)k - su.s0[2];
                for (int x = lo; x <= hi; ++x) {
                    const float dx = (float)x - su.s0[0];
                    const float yx = fmaf(M[0], dx, fmaf(M[1], dy, fmaf(M[2], dz, su.t0[0])));
                    const float yy = fmaf(M[3], dx, fmaf(M[4], dy, fmaf(M[5], dz, su.t0[1])));
                    const float yz = fmaf(M[6], dx, fmaf(M[7], dy, fmaf(M[8], dz, su.t0[2])));
                    const size_t idx = ((size_t)k * ny + j) * nx + x;
                    if (dvf) {
                        dvf[3 * idx] = yx - (float)x;
                        dvf[3 * idx + 1] = yy - (float)j;
                        dvf[3 * idx + 2] = yz - (float)k;
                    }
                    if (pull) {
                        const int mx = (int)fminf(fmaxf(rintf(yx), 0.0f), (float)(nx - 1));
                        const int my = (int)fminf(fmaxf(rintf(yy), 0.0f), (float)(ny - 1));
                        const int mz = (int)fminf(fmaxf(rintf(yz), 0.0f), (float)(nz - 1));
                        const int lb = lab_oth[((size_t)mz * ny + my) * nx + mx];
                        if (warped) warped[idx] = (uint8_t)lb;
                        if (!labels) continue;
                        const int la = lab_own[idx];
                        if (la < n_labels) atomicAdd(&hist[la][0], 1ull);
                        if (lb < n_labels) atomicAdd(&hist[lb][1], 1ull);
                        if (la == lb && la < n_labels) atomicAdd(&hist[la][2], 1ull);
                    }
                }
            }
        }
        __syncwarp();
    }
    if (labels) {
        __syncthreads();
        for (int i = threadIdx.x; i < n_labels * 3; i += blockDim.x) {
            const unsigned long long v = (&hist[0][0])[i];
            if (v) atomicAdd(counts + i, v);
        }
    }
}

}  // namespace

int dvf_max_labels() { return kMaxLabels; }

cudaError_t launch_dvf(const DevProblem *dp, const DevProblem &hp, const float *src, const float *tgt, int side,
                       float *dvf, const uint8_t *lab_own, const uint8_t *lab_oth, int n_labels,
                       unsigned long long *counts, uint8_t *warped, cudaStream_t st)
{
    const size_t N = (size_t)hp.nx * hp.ny * hp.nz;
    cudaError_t e = cudaSuccess;
    if (dvf) e = cudaMemsetAsync(dvf, 0xFF, 3 * N * sizeof(float), st);        // all-ones words are NaN
    if (e == cudaSuccess && counts) e = cudaMemsetAsync(counts, 0, 3 * (size_t)n_labels * sizeof(*counts), st);
    if (e == cudaSuccess && warped) e = cudaMemsetAsync(warped, 0xFF, N, st);           // 255: in no copy
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::min<long long>((hp.n_tets + kDvfWarps - 1) / kDvfWarps, 65535);
    k_dvf<<<blocks, kDvfWarps * 32, 0, st>>>(dp, src, tgt, side, dvf, lab_own, lab_oth, n_labels, counts, warped);
    return cudaGetLastError();
}

}  // namespace morea
