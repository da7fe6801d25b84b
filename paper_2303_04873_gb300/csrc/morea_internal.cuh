// Internal device-side structures and launch wrappers of libmorea.
// Not part of the public ABI (include/morea.h).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/morea.h"

namespace morea {

constexpr int kMaxGroups = 8;
constexpr int kBlock = 256;

// Everything a kernel needs to know about one registration problem.  Lives in
// device memory (one per problem) so batched launches can mix problems.
struct DevProblem {
    int nx, ny, nz, dtype;
    int kbits, S, H, h_mode;
    int g_mode, G, n_points, n_tets;
    float r, inv_r;
    int n_guid, cshift;
    float wgt[kMaxGroups];           // |C^k| / |G| per guidance group
    const void *img[2];              // [0] source image I_s, [1] target image I_t
    const float *dmap[2];            // [G][N] distance maps of the source / target contours
    const uint8_t *band[2];          // [N] bit g set where dmap[side][g] < r
    const int4 *tets;                // positively oriented topology
    const float *cdelta;             // elasticity factor per tet
    const int4 *gq[2];               // snapped guidance points per side
    const float4 *gp[2];             // raw guidance points per side
    const int *cell_start[2];        // guidance-point buckets (8^3-voxel cells), CSR
    const int *cell_pts[2];
    int cgx, cgy, cgz, max_sol;
    const int4 *slot_q;              // [max_sol][2][V] snapped coordinates of each slot
    morea_tet_record *cache;         // [max_sol][T]
    morea_totals *totals;            // [max_sol]
    unsigned int *status;            // device status word
};

// One (solution or request, tet) work unit with both copies' snapped vertices.
struct __align__(16) WorkEntry {
    int req, slot, tet, prob;
    int4 q[2][4];                    // [mesh: 0 source, 1 target][vertex]
};

// Per (entry, side) rasterisation set-up, written by the tet pass.
// Face f of the own copy: g_f . P + c_f + tie_f > 0 for P strictly inside
// after the symbolic perturbation.  For voxel rows (j, k) of the own image,
// with dj = j - jlo, dk = k - klo:   A_f i + B00_f + By_f dj + Bz_f dk > 0.
struct __align__(16) RasterSetup {
    long long ax[4], by[4], bz[4], b00[4];
    long long ct[4];                 // c_f + tie_f (for arbitrary snapped points)
    float e0[4], ey[4], ez[4];       // float estimate of the root -B/A in voxel index
    float M[9];                      // affine map own -> other, row-major
    float s0[3], t0[3];              // vertex 0 of the own / other copy, voxel units
    int ilo, ihi, jlo, jhi, klo, khi;  // voxel-centre index range of the bounding box
    int qlo[3], qhi[3];                // snapped bounding box
    int valid, pad;
};

struct __align__(16) RasterOut {
    float e_img, e_guid;
    int n_vox, n_gp;
};

struct __align__(16) TetOut {
    float e_mag;
    unsigned int folded;
    unsigned long long sev;
};

struct ReqInfo {
    int base, count, err, slot, nchg, pad0, pad1, pad2;
};

// ---------------------------------------------------------------------------
// launch wrappers (k_tet.cu, k_raster.cu)
// ---------------------------------------------------------------------------

cudaError_t launch_snap_slots(const DevProblem *dp, const DevProblem &hp, int n_sol, const int *slot,
                              const float *src, const float *tgt, int4 *slot_q, int max_sol,
                              cudaStream_t st);
cudaError_t launch_full_entries(const DevProblem *dp, const DevProblem &hp, int n_sol, const int *slot,
                                WorkEntry *entries, RasterSetup *setup, TetOut *tout, cudaStream_t st);
cudaError_t launch_raster(const DevProblem *probs, const DevProblem &hp, const WorkEntry *entries,
                          const RasterSetup *setup, RasterOut *rout, const int *n_entries_dev,
                          int n_entries_host, int grid, cudaStream_t st);
cudaError_t launch_reduce_full(const DevProblem *dp, const DevProblem &hp, int n_sol, const int *slot,
                               const TetOut *tout, const RasterOut *rout, double *obj, uint8_t *folded,
                               double *severity, cudaStream_t st);
cudaError_t launch_partial_entries(const DevProblem *dp, const DevProblem &hp, int n_req, const int *slot,
                                   const int *chg_off, const int *chg_pts, const float *chg_src,
                                   const float *chg_tgt, int max_sol, int max_changed,
                                   const int *v2t_off, const int *v2t_idx, WorkEntry *entries,
                                   RasterSetup *setup, TetOut *tout, int cap_entries, int *counter,
                                   ReqInfo *rinfo, int *req_chg_pts, int4 *req_chg_q, cudaStream_t st);
cudaError_t launch_partial_finalize(const DevProblem *dp, const DevProblem &hp, int n_req,
                                    const ReqInfo *rinfo, const WorkEntry *entries, const TetOut *tout,
                                    const RasterOut *rout, morea_totals *delta, double *obj,
                                    uint8_t *folded, double *severity, cudaStream_t st);
cudaError_t launch_partial_commit(const DevProblem *dp, const DevProblem &hp, int n_req,
                                  const uint8_t *accept, const ReqInfo *rinfo, const WorkEntry *entries,
                                  const TetOut *tout, const RasterOut *rout, const morea_totals *delta,
                                  const int *req_chg_pts, const int4 *req_chg_q, int max_changed,
                                  const int *counter, int cap, int4 *slot_q, cudaStream_t st);
cudaError_t launch_check_folds(const DevProblem *dp, const DevProblem &hp, int n_sol, const float *src,
                               const float *tgt, uint8_t *folded, double *severity, cudaStream_t st);
cudaError_t launch_gather_records(const DevProblem &hp, int n_sol, const int *slot,
                                  morea_tet_record *out, cudaStream_t st);
cudaError_t launch_gather_totals(const DevProblem &hp, int n_sol, const int *slot, morea_totals *out,
                                 cudaStream_t st);
cudaError_t launch_distance_maps(const DevProblem &hp, const float4 *pts, const int *goff, float *dmap,
                                 uint8_t *band, cudaStream_t st);

cudaError_t launch_count_visits(const RasterOut *rout, const int *n_entries_dev, int n_entries_host,
                                unsigned long long *visits, cudaStream_t st);

int sm_count();
size_t partial_smem_bytes(int n_tets, int max_changed);

}  // namespace morea
