// Internal device-side structures and launch wrappers of libmorea.
// Not part of the public ABI (include/morea.h).
#pragma once

#include <cstddef>

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/morea.h"

namespace morea {

constexpr int kMaxGroups = 8;
constexpr int kBlock = 256;

constexpr int kMaxBatch = 64;

// Completion clock of a batched evaluation (morea_batch_*), per problem of
// the batch: its items counted as the passes finish them, and the
// %globaltimer (ns) at which its last image-pass item, its last guidance item
// and its last objective reduction finished; t0 is stamped by the first
// kernel of the batch.
struct BatchClock {
    unsigned long long t0;
    unsigned long long t_raster[kMaxBatch], t_guid[kMaxBatch], t_reduce[kMaxBatch];
    int raster_done[kMaxBatch], raster_total[kMaxBatch];
    int guid_done[kMaxBatch], guid_total[kMaxBatch];
    int reduce_done[kMaxBatch];
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Everything a kernel needs to know about one registration problem.  Lives in
// device memory (one per problem) so batched launches can mix problems.
struct DevProblem {
    int nx, ny, nz, dtype;
    int kbits, S, H, h_mode;
    int estimator;                   // morea_estimator
    float rate;                      // sampled estimator: points per voxel^3
    int g_mode, G, n_points, n_tets;
    float r, inv_r;
    int n_guid, cshift;
    float wgt[kMaxGroups];           // |C^k| / |G| per guidance group
    const void *img[2];              // [0] source image I_s, [1] target image I_t
    const void *quad[2];             // padded quad copies (quad_cells), at the element of cell (0, 0, 0)
    const float *dmap[2];            // [G][N] distance maps of the source / target contours
    const uint8_t *band[2];          // [N] bit g set where dmap[side][g] < r
    const short2 *bandrow[2];        // [nz*ny] x-range of band voxels in each image row (empty: x > y)
    const int *band_start[2];        // [nz*ny + 1] CSR of the band voxels of each image row
    const int2 *band_rec[2];         // per band voxel: x | band bits << 16, and the bits of its own distance
                                     // to the lowest band group; ascending x within a row
    const short *band_rank[2];       // [N] band voxels before x in the same image row
    const uint8_t *bandd[2];         // [N] band bits OR-ed over the 2x2x2 cell at each voxel (sampled)
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
    BatchClock *clock;               // batched evaluation only (the batch's copy): completion clock, else NULL
};

// One (solution or request, tet) work unit with both copies' snapped vertices.
struct __align__(16) WorkEntry {
    int req, slot, tet, prob;
    int4 q[2][4];                    // [mesh: 0 source, 1 target][vertex]
};

// One face f of a tet copy as a function of the voxel row (j, k): the voxel
// centre (i, j, k) is inside w.r.t. f iff  ax i + b00 + by dj + bz dk > 0
// (dj = j - jlo, dk = k - klo; integers, simulation-of-simplicity tie bit
// folded into b00).  e0 + ey dj + ez dk estimates the root -B/A in FP32 to
// within |tol| for every row of the bounding box (a rigorous bound); tol
// carries the sign of ax, and is +infinity when ax = 0.
struct __align__(16) FaceRow {
    long long ax, b00, by, bz;
    float e0, ey, ez, tol;
};

// Per (entry, side) rasterisation set-up, written by the tet pass.
struct __align__(16) RasterSetup {
    FaceRow f[4];
    long long ct[4];                 // c_f + tie_f (inside test of arbitrary snapped points)
    float M[9];                      // affine map own -> other, row-major, voxel units
    float s0[3];                     // vertex 0 of the own copy
    float t0[3];                     // vertex 0 of the other copy
    int valid;                         // bit 0: orientation > 0; bit 1: the other copy lies
                                       // strictly inside (-1, n) per axis (the padded quad copy
                                       // needs no sample clamping)
    int ilo, ihi, jlo, jhi, klo, khi;  // voxel-centre index range of the bounding box
    int qlo[3], qhi[3];                // snapped bounding box
};

// k_raster reads the set-up with vector loads at these offsets
static_assert(sizeof(FaceRow) == 48, "FaceRow layout");
static_assert(offsetof(RasterSetup, M) % 16 == 0, "M must start a 16-byte word");
static_assert(offsetof(RasterSetup, s0) == offsetof(RasterSetup, M) + 36, "M[8], s0 share a word");
static_assert(offsetof(RasterSetup, t0) % 16 == 0, "t0 must start a 16-byte word");
static_assert(offsetof(RasterSetup, valid) == offsetof(RasterSetup, t0) + 12, "t0, valid share a word");
static_assert(offsetof(RasterSetup, ilo) % 16 == 0, "ilo..jhi form one int4");
static_assert(offsetof(RasterSetup, klo) % 8 == 0, "klo, khi form one int2");

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

// One problem's share of a batched full evaluation (morea_batch_*): its
// inputs and outputs and where its work sits in the batch's flattened lists.
struct BatchProb {
    const float *src, *tgt;          // [n_sol][V][3]
    double *obj;                     // [n_sol][3]
    uint8_t *folded;                 // [n_sol]
    double *severity;                // [n_sol] or NULL
    long long vert_off;              // first (solution, vertex) of the problem
    long long entry_off;             // first (solution, tet) entry of the problem
    int sol_off;                     // first solution of the problem
    int n_sol;
};

// Passed by value to the batch kernels (kernel parameters are copied at
// launch, so no host buffer has to outlive the call or a captured graph).
struct BatchTable {
    int n;
    int pad;
    long long total_verts, total_entries;
    int total_sols;
    int pad2;
    BatchProb p[kMaxBatch];
};

// ---------------------------------------------------------------------------
// launch wrappers (k_tet.cu, k_raster.cu, k_batch.cu)
// ---------------------------------------------------------------------------

cudaError_t launch_snap_slots(const DevProblem *dp, const DevProblem &hp, int n_sol, const int *slot,
                              const float *src, const float *tgt, int4 *slot_q, int max_sol,
                              cudaStream_t st);
cudaError_t launch_full_entries(const DevProblem *dp, const DevProblem &hp, int n_sol, const int *slot,
                                WorkEntry *entries, RasterSetup *setup, TetOut *tout, cudaStream_t st);
// rqueue (or NULL): the image pass's queue; the entry pass then also writes
// the order of its items (largest copies first, see kQueueList) and the
// image pass takes the items in that order.
cudaError_t launch_entry_work(const DevProblem *dp, const WorkEntry *entries, RasterSetup *setup, TetOut *tout,
                              const int *n_entries_dev, int n_entries_host, int *rqueue, cudaStream_t st);
// Quad copy of an image: per cell (x, y, z), -1 <= x < nx, -1 <= y < ny,
// -1 <= z <= nz, the values at (x, y), (x+1, y), (x, y+1), (x+1, y+1) of
// z-plane z, each index clamped into the image (so the padding repeats the
// edge values).  Element (x, y, z) sits at (z (ny+1) + y) (nx+1) + x from the
// element of cell (0, 0, 0), which lies quad_origin elements into the array.
inline long long quad_cells(int nx, int ny, int nz) { return (long long)(nx + 1) * (ny + 1) * (nz + 2); }
inline long long quad_origin(int nx, int ny) { return (long long)(nx + 1) * (ny + 2) + 1; }
// builds the quad copy of one side into `quad` (quad_cells elements)
cudaError_t launch_build_quads(const DevProblem &hp, int side, void *quad, cudaStream_t st);
cudaError_t launch_band_rows(const DevProblem &hp, int side, short2 *bandrow, cudaStream_t st);
// fills the distance word of the band records of one side (x and bits set by the host)
cudaError_t launch_band_records(const DevProblem &hp, int side, int2 *rec, cudaStream_t st);
// image pass (+ continuous guidance pass); bandrows: [2 * entries][kBandRowsPerItem] scratch
constexpr int kBandRowsPerItem = 128;
// chunk > 0 selects the atomic work queue.  queue: kQueueList device counters
// (the first kQueueOrderBig reset by launch_raster, the large-item count by
// the caller before the entry pass), then the list of the (entry, side)
// items that have band rows
// (continuous guidance; capacity 2 * n_entries_host), then the list of the
// large items the image pass takes first (capacity 2 * n_entries_host).
constexpr int kQueueRaster = 0;      // work counter of the image pass
constexpr int kQueueGuidance = 1;    // work counter of the guidance pass
constexpr int kQueueListCount = 2;   // items listed for the guidance pass
constexpr int kQueueOrderBig = 3;    // large items listed for the image pass to take first
constexpr int kQueueList = 8;        // first list entry (32-byte aligned)
// A copy whose bounding box holds at least this many voxel centres is an
// item the ordered image pass takes first.
constexpr int kBigItemVoxels = 32768;
inline size_t queue_ints(long long cap_entries, bool continuous)
{
    (void)continuous;
    return kQueueList + 4 * (size_t)cap_entries;
}
// The sampled estimator (k_sample.cu): Sobol direction numbers into constant
// memory (once per device), the dilated band masks, and the image pass.
cudaError_t sample_setup(cudaStream_t st);
cudaError_t launch_band_dilate(const DevProblem &hp, const uint8_t *band, uint8_t *out, cudaStream_t st);
cudaError_t launch_sample(const DevProblem *probs, const DevProblem &hp, const WorkEntry *entries,
                          const RasterSetup *setup, RasterOut *rout, const int *n_entries_dev, int n_entries_host,
                          int grid, int chunk, int *queue, cudaStream_t st);
// Displacement field and label overlap of one solution (k_dvf.cu).
cudaError_t launch_slot_objectives(const DevProblem *dp, int n_sol, const int *slot, double *obj, uint8_t *folded,
                                  double *severity, cudaStream_t st);
size_t sample_elements_bytes(int n_clusters, int n_elements);
cudaError_t launch_sample_elements(int V, int n_pop, const float *src, const float *tgt, int C, int csize,
                                   const int *members, int m, const int *elements, const uint8_t *fixed,
                                   const float *cmult, int n_req, const int *req_sol, const int *req_cluster,
                                   const int *req_elem, const float *z, void *work, float *new_src, float *new_tgt,
                                   cudaStream_t st);
size_t init_smem_bytes(int n_points, int n_kernels);
cudaError_t launch_init(const DevProblem *dp, const DevProblem &hp, int n_sol, float *src, float *tgt,
                        const uint8_t *fixed, int n_kernels, const float *kernels, int max_rounds, int *rounds,
                        cudaStream_t st);
int dvf_max_labels();
// Elasticity factors from a tissue mask (k_tissue.cu): per tet, the mean of
// factor[mask] over the voxel centres of its positively oriented reference
// copy; tets with no voxel centre keep their value in cdelta.
constexpr int kMaxTissueLabels = 64;
cudaError_t launch_tissue_factors(const DevProblem &hp, const int4 *tets, const int4 *qref, const uint8_t *mask,
                                  const double *factor, int n_labels, float *cdelta, cudaStream_t st);
cudaError_t launch_dvf(const DevProblem *dp, const DevProblem &hp, const float *src, const float *tgt, int side,
                       float *dvf, const uint8_t *lab_own, const uint8_t *lab_oth, int n_labels,
                       unsigned long long *counts, uint8_t *warped, cudaStream_t st);
// Repair of folded solutions (k_repair.cu), one warp per solution.
cudaError_t launch_repair(const DevProblem *dp, const DevProblem &hp, const int *v2t_off, const int *v2t_idx,
                          int n_sol, float *src, float *tgt, const float *noise, int max_points, double scale, const uint8_t *fixed,
                          int *moved, double *severity, cudaStream_t st);
cudaError_t launch_raster(const DevProblem *probs, const DevProblem &hp, const WorkEntry *entries,
                          const RasterSetup *setup, RasterOut *rout, int2 *bandrows, const int *n_entries_dev,
                          int n_entries_host, int grid, int chunk, int *queue, bool ordered, BatchClock *clock,
                          cudaStream_t st);
cudaError_t launch_reduce_full(const DevProblem *dp, const DevProblem &hp, int n_sol, const int *slot,
                               const TetOut *tout, const RasterOut *rout, double *obj, uint8_t *folded,
                               double *severity, cudaStream_t st);
cudaError_t launch_partial_entries(const DevProblem *dp, const DevProblem &hp, int n_req, const int *slot,
                                   const int *chg_off, const int *chg_pts, const float *chg_src,
                                   const float *chg_tgt, int max_sol, int max_changed,
                                   const int *v2t_off, const int *v2t_idx, WorkEntry *entries,
                                   RasterSetup *setup, TetOut *tout, int cap_entries, int *counter,
                                   ReqInfo *rinfo, int *req_chg_pts, int4 *req_chg_q, int *rqueue,
                                   cudaStream_t st);
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

cudaError_t launch_batch_snap(const DevProblem *probs, const BatchTable &tb, cudaStream_t st);
cudaError_t launch_batch_entries(const DevProblem *probs, const BatchTable &tb, WorkEntry *entries, cudaStream_t st);
cudaError_t launch_batch_reduce(const DevProblem *probs, const BatchTable &tb, const TetOut *tout,
                                const RasterOut *rout, cudaStream_t st);

cudaError_t launch_partial_features(const DevProblem *dp, int n_req, const int *slot, const int *chg_off,
                                    const int *chg_pts, const float *chg_src, const float *chg_tgt, float *out,
                                    cudaStream_t st);

int sm_count();
size_t partial_smem_bytes(int n_tets, int max_changed);
// Snapping grid of reading R1 for an image box and tet count: the requested
// k if it keeps coordinates below 2^16 and the exact severity sum in 64
// bits, else -1; 0 picks the largest such k <= 8 (morea_abi.cu).
int choose_subvoxel_bits(int requested, int nx, int ny, int nz, long long n_tets);

}  // namespace morea
