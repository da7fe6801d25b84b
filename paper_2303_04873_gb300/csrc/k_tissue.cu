// Elasticity factor of each tet from a tissue mask (App. A.1): the factor of
// a tet weights the tissues it overlaps, c = sum_k frac_k f_k +
// (1 - sum_k frac_k) f_0, with frac_k the share of the tet in tissue k and
// label 0 the background.  The share is taken on the voxel grid: the voxel
// centres of the tet's reference copy by the exact association of reading
// R3, counted per label of the mask.  Then c = sum_l count_l f_l / sum_l
// count_l, summed in FP64 in label order.
//
// One warp per tet: lane 0 builds the copy's rasterisation set-up in shared
// memory, the lanes take the rows of its bounding box, and the label counts
// go to a per-warp histogram in shared memory.  Runs once, at problem
// creation.
#include <algorithm>

#include "image_ops.cuh"

namespace morea {

namespace {

constexpr int kTisWarps = 8;

__global__ void __launch_bounds__(kTisWarps * 32) k_tissue(DevProblem P, const int4 *__restrict__ tets,
                                                           const int4 *__restrict__ qref,
                                                           const uint8_t *__restrict__ mask,
                                                           const double *__restrict__ factor, int n_labels,
                                                           float *__restrict__ cdelta)
{
    __shared__ RasterSetup sus[kTisWarps];
    __shared__ unsigned hist[kTisWarps][kMaxTissueLabels];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    RasterSetup &su = sus[warp];
    unsigned *h = hist[warp];
    const int nx = P.nx, ny = P.ny;
    for (int t = blockIdx.x * kTisWarps + warp; t < P.n_tets; t += gridDim.x * kTisWarps) {
        for (int l = lane; l < kMaxTissueLabels; l += 32) h[l] = 0u;
        if (lane == 0) {
            const int4 tv = tets[t];
            const int4 own[4] = {qref[tv.x], qref[tv.y], qref[tv.z], qref[tv.w]};
            make_setup(own, own, P, su);
        }
        __syncwarp();
        if (su.valid & 1) {
            const int ilo = su.ilo, ihi = su.ihi, jlo = su.jlo, klo = su.klo;
            const int nyb = su.jhi - jlo + 1, nzb = su.khi - klo + 1;
            const int n_rows = (ilo <= ihi && nyb > 0 && nzb > 0) ? nyb * nzb : 0;
            for (int r = lane; r < n_rows; r += 32) {
                const int dk = r / nyb, dj = r - dk * nyb;
                int lo, hi;
                row_interval<false>(su.f, dj, dk, ilo, ihi, lo, hi);   // set-up in shared memory
                const size_t row = ((size_t)(klo + dk) * ny + (jlo + dj)) * nx;
                for (int x = lo; x <= hi; ++x) atomicAdd(&h[mask[row + x]], 1u);
            }
        }
        __syncwarp();
        if (lane == 0) {
            long long n = 0;
            double s = 0.0;
            for (int l = 0; l < n_labels; ++l) {
                n += h[l];
                s += (double)h[l] * factor[l];
            }
            if (n > 0) cdelta[t] = (float)(s / (double)n);
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_tissue_factors(const DevProblem &hp, const int4 *tets, const int4 *qref, const uint8_t *mask,
                                  const double *factor, int n_labels, float *cdelta, cudaStream_t st)
{
    const int blocks = (int)std::min<long long>((hp.n_tets + kTisWarps - 1) / kTisWarps, 65535);
    k_tissue<<<blocks, kTisWarps * 32, 0, st>>>(hp, tets, qref, mask, factor, n_labels, cdelta);
    return cudaGetLastError();
}

}  // namespace morea
