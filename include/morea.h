/*
 * morea.h -- C ABI of libmorea, a GB300 (sm_103a) evaluator for the
 * objectives and the fold constraint of MOREA (Andreadis, Bosman,
 * Alderliesten, "MOREA: a GPU-accelerated Evolutionary Algorithm for
 * Multi-Objective Deformable Registration of 3D Medical Images", GECCO 2023,
 * arXiv 2303.04873).
 *
 * A registration solution is a pair of tetrahedral meshes with one shared
 * topology: one mesh on the source image I_s, one on the target image I_t
 * (the dual-dynamic model, Sec. 1 and Sec. 4.2.1).  Each tet defines an
 * affine map T between its source and target copies and the inverse map T'.
 * libmorea evaluates, for a population of such solutions,
 *   obj[0] f_intensity  (Sec. 4.1.2, equations for f_intensity and h),
 *   obj[1] f_magnitude  (Sec. 4.1.1, f_magnitude equation; App. A.1),
 *   obj[2] f_guidance   (Sec. 4.1.3, equations for f_guidance and g; App. A.3),
 * and the fold constraint (Sec. 4.1.4; App. A.4), fully or by partial
 * re-evaluation of the tets that depend on changed points (Sec. 1;
 * Sec. 4.2.1).  All three objectives are minimised.
 *
 * Conventions
 *   - Images are [nz][ny][nx], x fastest.  Coordinates are voxel-index
 *     units: voxel (i, j, k) has its centre at (i, j, k); the image box is
 *     [-0.5, n - 0.5] per axis.  Points are (x, y, z) float triples.
 *   - Every coordinate is clamped to the image box and snapped, round half
 *     to even, onto a grid of 2^-k voxel (k = subvoxel_bits).  On that grid
 *     orientation determinants are exact, so coverage counts and fold flags
 *     are exact integers.
 *   - A voxel centre belongs to a tet iff it is inside the tet after the
 *     symbolic perturbation (e, e^2, e^3), e -> 0+.  On a conforming,
 *     box-filling, unfolded mesh every voxel centre is counted exactly once.
 *     A folded tet copy (orientation <= 0) is not rasterised.
 *   - "stream" is a cudaStream_t (NULL = legacy default stream).  Every
 *     evaluation call only enqueues work on that stream: it does not
 *     synchronise and does not allocate memory.  All memory a problem needs
 *     is allocated by morea_create_problem.
 *   - Pointers documented "device" must be device (or managed) memory of the
 *     current device; "host" pointers are read before the call returns.
 *     The caller owns every pointer it passes; the handle owns its copies.
 *   - Argument errors are found on the host before anything is enqueued and
 *     return MOREA_EINVAL with nothing launched.  Errors that only the GPU
 *     can see (a point id out of range in a partial request, a request longer
 *     than max_changed, a scratch overflow) set bits in a device status word
 *     of the problem; the request's outputs become NaN / folded = 1, and
 *     morea_device_status returns and clears the word.  No kernel traps.
 */
#ifndef MOREA_H
#define MOREA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum morea_status {
    MOREA_OK = 0,
    MOREA_EINVAL = 1,      /* invalid argument or problem description */
    MOREA_ENOMEM = 2,      /* device or host allocation failed (create only) */
    MOREA_ECUDA = 3,       /* a CUDA runtime call failed */
    MOREA_ETIMEOUT = 4,    /* a bounded device-side wait gave up */
    MOREA_ENOTIMPL = 5,    /* option not implemented */
    MOREA_EDEVICE = 6      /* the device status word reported bad input */
} morea_status;

typedef enum morea_dtype { MOREA_F32 = 0, MOREA_F16 = 1 } morea_dtype;

/* h of Sec. 4.1.2.  PLAIN_SSD: (a - b)^2.  MOREA_FG: the printed case split:
 * (a - b)^2 if a > 0 and b > 0; 0 if a == 0 and b == 0; 1 otherwise, with
 * a the stored voxel value and b the trilinear sample of the other image. */
typedef enum morea_hmode { MOREA_H_PLAIN_SSD = 0, MOREA_H_MOREA_FG = 1 } morea_hmode;

/* CONTINUOUS: the distance-map formulation of Sec. 4.1.3 / App. A.3.
 * PAIR_TRANSFER: the exact measure of the prior work described in App. A.3:
 * mean of |T(g_s) - g_t|^2 and |T'(g_t) - g_s|^2 over located points.
 * OFF: f_guidance = 0. */
typedef enum morea_gmode {
    MOREA_G_CONTINUOUS = 0, MOREA_G_PAIR_TRANSFER = 1, MOREA_G_OFF = 2
} morea_gmode;

/* Which points of a tet copy enter f_intensity and f_guidance.
 * VOXELS: the voxel centres inside the copy, made exact by a symbolic
 * perturbation (the association the paper's App. A.2 starts from, made
 * watertight).  SAMPLED: the paper's own estimator (App. A.2): per copy
 * N = floor(rate * volume + 1/2) points (capped at 2^24), uniform in
 * barycentric coordinates from -log of a 4-D Sobol sequence (Gray-code
 * order, Joe-Kuo direction numbers) whose 32-bit coordinates are XOR-shifted
 * by values derived from the copy's snapped coordinates (FNV-1a over the 12
 * coordinates as little-endian int32, then the first four splitmix64
 * outputs, high 32 bits), so a copy always gets the same points; both
 * images and the guidance maps are sampled trilinearly there.  SAMPLED
 * requires h_mode PLAIN_SSD and g_mode CONTINUOUS or OFF. */
typedef enum morea_estimator { MOREA_EST_VOXELS = 0, MOREA_EST_SAMPLED = 1 } morea_estimator;

/* Bits of the device status word. */
#define MOREA_DEV_BAD_POINT     0x1u   /* partial request names a point id out of range */
#define MOREA_DEV_TOO_MANY      0x2u   /* partial request longer than max_changed / bad offsets */
#define MOREA_DEV_DUPLICATE     0x4u   /* partial request lists a point twice */
#define MOREA_DEV_OVERFLOW      0x8u   /* affected-tet scratch overflow */
#define MOREA_DEV_BAD_SLOT      0x10u  /* slot index out of range */
#define MOREA_DEV_TIMEOUT       0x20u  /* bounded wait gave up */

typedef struct morea_problem morea_problem;            /* opaque handle */

/* Problem description (Sec. 4.1).  Read during morea_create_problem only. */
typedef struct morea_problem_desc {
    int32_t nx, ny, nz;            /* image extent, each >= 2 */
    int32_t dtype;                 /* morea_dtype of both images */
    const void *image_s;           /* source image I_s, [nz][ny][nx], host or device */
    const void *image_t;           /* target image I_t, same layout */
    int32_t n_points, n_tets;      /* V >= 4, T >= 1 */
    const int32_t *tets;           /* host [T][4] vertex ids, shared topology */
    const float *ref_points;       /* host [V][3] initial mesh: gives the reference signs */
    const int32_t *tet_label;      /* host [T] tissue label per tet, or NULL (all 0) */
    const double *tissue_factor;   /* host [n_labels] elasticity factor per label, or NULL (1.0) */
    int32_t n_labels;
    int32_t n_guid;                /* number of guidance point pairs (>= 0) */
    const float *guid_s;           /* host [n_guid][3] contour points on I_s */
    const float *guid_t;           /* host [n_guid][3] corresponding points on I_t */
    const int32_t *guid_group;     /* host [n_guid] contour-group id in [0, 8), or NULL (all 0) */
    double trunc_radius;           /* guidance truncation radius r in voxels; <= 0: 0.025 * nx */
    int32_t h_mode;                /* morea_hmode */
    int32_t g_mode;                /* morea_gmode */
    int32_t subvoxel_bits;         /* k in [2, 14] with max(nx, ny, nz) * 2^k <= 65536; 0: 8 */
    int32_t max_solutions;         /* number of cache slots (solutions kept resident) >= 1 */
    int32_t max_requests;          /* largest n_req of morea_eval_partial (0: max_solutions) */
    int32_t max_changed;           /* largest changed-point count of one request (0: 64) */
    int32_t estimator;             /* morea_estimator (0: VOXELS) */
    float sampling_rate;           /* SAMPLED: points per voxel^3 of tet volume (<= 0: 1.0) */
    const uint8_t *tissue_mask;    /* host [nz][ny][nx] tissue label of each voxel of I_s, or NULL.
                                    * Given (with tissue_factor, labels < n_labels <= 64), the
                                    * elasticity factor of a tet is the mean of tissue_factor over
                                    * the labels of the voxel centres in its reference copy (exact
                                    * association): sum_k frac_k f_k + (1 - sum_k frac_k) f_0 with
                                    * label 0 the background (App. A.1).  A tet that contains no
                                    * voxel centre keeps tissue_factor[tet_label]. */
} morea_problem_desc;

/* Per-(slot, tet) summands kept by the handle (what a partial evaluation
 * subtracts and adds).  Index 0 = source side (voxels of I_s in the source
 * copy), 1 = target side. */
typedef struct morea_tet_record {
    float e_img[2];       /* sum of h over the tet copy's voxel centres */
    float e_guid[2];      /* continuous: weighted sum of g terms; pair: sum of squared transfer errors */
    int32_t n_vox[2];     /* voxel centres associated with the tet copy (exact) */
    int32_t n_gp[2];      /* guidance points located in the copy (pair mode) */
    float e_mag;          /* c_delta * sum over the 10 edges of (|e_s| - |e_t|)^2 */
    uint32_t folded;      /* bit 0: source copy folded, bit 1: target copy folded */
    uint64_t sev;         /* sum of |orient| over folded copies (integer, 6 * 2^3k * voxel^3) */
} morea_tet_record;

/* Per-slot totals over all tets (FP64 sums, exact integer counts). */
typedef struct morea_totals {
    double s_img, s_guid, s_mag;
    int64_t n_vox, n_gp, n_folded;
    uint64_t sev;
    int64_t reserved;
} morea_totals;

/* Create a problem: validates the description, copies the images to the
 * device, orients every tet positively against ref_points (a zero reference
 * volume is MOREA_EINVAL), builds the vertex-to-tet adjacency, computes the
 * guidance distance maps (Sec. 4.1.3) and allocates the per-slot caches and
 * all scratch.  Synchronises `stream` before returning.
 * On error *out is NULL and nothing is leaked. */
morea_status morea_create_problem(const morea_problem_desc *desc, void *stream,
                                  morea_problem **out);

/* Frees everything the handle owns (synchronises the device first).  NULL is a no-op. */
morea_status morea_destroy_problem(morea_problem *p);

/* Full evaluation (Sec. 4.1) of n_sol solutions.
 *   slot      device [n_sol] cache slot of each solution in [0, max_solutions),
 *             distinct within a call, or NULL for slots 0..n_sol-1
 *   src_pts   device [n_sol][V][3] source-mesh points
 *   tgt_pts   device [n_sol][V][3] target-mesh points
 *   obj       device [n_sol][3] out: f_intensity, f_magnitude, f_guidance
 *   folded    device [n_sol] out: 1 if any tet copy of either mesh is folded
 *   severity  device [n_sol] out, or NULL: sum of |signed volume| (voxel^3) of folded copies
 * The slots' coordinates, per-tet records and totals are replaced, so later
 * partial evaluations start from these solutions. */
morea_status morea_eval_full(morea_problem *p, int32_t n_sol, const int32_t *slot,
                             const float *src_pts, const float *tgt_pts,
                             double *obj, uint8_t *folded, double *severity, void *stream);

/* Partial evaluation (Sec. 1; Sec. 4.2.1): request r moves the points
 * chg_pts[chg_off[r] .. chg_off[r+1]) of the solution in slot[r] to
 * chg_src / chg_tgt (absolute coordinates, aligned with chg_pts).  Only
 * the tets incident to a moved point are re-evaluated; the result is the
 * slot's totals plus the sum over those tets of (new - cached).
 *   slot      device [n_req]
 *   chg_off   device [n_req + 1], non-decreasing, chg_off[0] = 0
 *   chg_pts   device [chg_off[n_req]] point ids, distinct within a request,
 *             at most max_changed per request
 *   chg_src   device [chg_off[n_req]][3]
 *   chg_tgt   device [chg_off[n_req]][3]
 *   obj, folded, severity  as in morea_eval_full, per request (severity may be NULL)
 *   commit    device [n_req] or NULL: nonzero commits the request into its
 *             slot right away (same as morea_commit_partial afterwards)
 * n_req <= max_requests.  Requests on the same slot are evaluated against
 * the slot's state before the call; if several of them are committed their
 * affected tets must be disjoint.  The scratch of this call stays valid for
 * morea_commit_partial until the next morea_eval_partial on the handle. */
morea_status morea_eval_partial(morea_problem *p, int32_t n_req, const int32_t *slot,
                                const int32_t *chg_off, const int32_t *chg_pts,
                                const float *chg_src, const float *chg_tgt,
                                double *obj, uint8_t *folded, double *severity,
                                const uint8_t *commit, void *stream);

/* Commit the requests of the last morea_eval_partial whose accept[r] is
 * nonzero (accept: device [n_req], n_req equal to that call's).  This is the
 * acceptance step of optimal mixing (Sec. 3): an accepted partial solution
 * replaces its parent in the slot. */
morea_status morea_commit_partial(morea_problem *p, int32_t n_req, const uint8_t *accept,
                                  void *stream);

/* Fold constraint only (Sec. 4.1.4; App. A.4) for n_sol solutions, without
 * touching any slot: folded [n_sol] and severity [n_sol] (may be NULL), device. */
morea_status morea_check_folds(morea_problem *p, int32_t n_sol, const float *src_pts,
                               const float *tgt_pts, uint8_t *folded, double *severity,
                               void *stream);

/* Copy the cached per-tet records of n_sol slots (device [n_sol], or NULL
 * for 0..n_sol-1) into out (device [n_sol][T]), tets in the problem's order. */
morea_status morea_read_records(morea_problem *p, int32_t n_sol, const int32_t *slot,
                                morea_tet_record *out, void *stream);

/* Copy the totals of n_sol slots into out (device [n_sol]). */
morea_status morea_read_totals(morea_problem *p, int32_t n_sol, const int32_t *slot,
                               morea_totals *out, void *stream);

/* Synchronise `stream`, return and clear the device status word (bits
 * MOREA_DEV_*) in *bits; returns MOREA_EDEVICE if any bit was set. */
morea_status morea_device_status(morea_problem *p, void *stream, uint32_t *bits);

/* Problem sizes after creation: n_points, n_tets, number of guidance
 * groups, truncation radius and subvoxel_bits in use (any output may be NULL). */
morea_status morea_problem_info(const morea_problem *p, int32_t *n_points, int32_t *n_tets,
                                int32_t *n_groups, double *trunc_radius, int32_t *subvoxel_bits);

/* ---- batched multi-problem evaluation (one launch per kernel for all) ---- */

typedef struct morea_batch morea_batch;                 /* opaque handle */

/* Maximum number of problems in one batch. */
#define MOREA_MAX_BATCH 64

/* Group n_problems (1..MOREA_MAX_BATCH) distinct problems created on the same
 * device with the same storage type, h_mode and g_mode, so that one launch of
 * each kernel evaluates all of them: the work entries of all problems form
 * one list that the image pass walks as a single persistent launch.
 * Allocates the batch's own scratch (sum over problems of max_solutions x
 * n_tets work entries).  The problems must outlive the batch; the batch
 * writes slots 0..n_sol[i]-1 of problem i. */
morea_status morea_batch_create(morea_problem *const *problems, int32_t n_problems, morea_batch **out);

/* Frees the batch's scratch and graph (not the problems).  NULL is a no-op. */
morea_status morea_batch_destroy(morea_batch *b);

/* Full evaluation (Sec. 4.1) of n_sol[i] solutions of every problem i of the
 * batch, as morea_eval_full with slots 0..n_sol[i]-1, with one launch per
 * kernel for the whole batch.  All pointer arguments are host arrays of
 * n_problems device pointers (severity may be NULL, or hold NULL entries).
 * Results are identical to per-problem morea_eval_full calls. */
morea_status morea_batch_eval_full(morea_batch *b, const int32_t *n_sol, const float *const *src_pts,
                                   const float *const *tgt_pts, double *const *obj,
                                   uint8_t *const *folded, double *const *severity, void *stream);

/* Record one morea_batch_eval_full with these arguments into a CUDA graph
 * held by the batch (replacing any previous one); `stream` must be a
 * non-default stream, used for the capture only.  The graph keeps the device
 * pointers and sizes given here and the launch shape in force now. */
morea_status morea_batch_capture(morea_batch *b, const int32_t *n_sol, const float *const *src_pts,
                                 const float *const *tgt_pts, double *const *obj,
                                 uint8_t *const *folded, double *const *severity, void *stream);

/* Launch the captured graph on `stream` (the evaluation reads the current
 * contents of the captured input buffers).  MOREA_EINVAL if none captured. */
morea_status morea_batch_replay(morea_batch *b, void *stream);

/* Per-problem completion times of the batch's last evaluation (direct or
 * replayed), in ms after its first kernel started, measured on the device
 * with %globaltimer (no events): records_ms[i] when the last image-pass or
 * guidance item of problem i finished (its per-tet records are final),
 * objectives_ms[i] when its last objective reduction finished.  Host arrays
 * [n_problems], either may be NULL; -1 for a problem whose evaluation did
 * not complete.  Synchronises the device.  The paper has no counterpart:
 * it measures the batching of several registration problems in one launch
 * sequence. */
morea_status morea_batch_latency(morea_batch *b, double *records_ms, double *objectives_ms);

/* Launch shape of the image and guidance passes, normally chosen by the
 * autotuner (paper_2303_04873_gb300.autotune): blocks_per_sm in [1, 64]
 * (grid = blocks_per_sm x SM count) and chunk in [0, 1024]: 0 = static
 * striding of (tet, side) items over warps, > 0 = warps take `chunk` items
 * at a time from an atomic work queue.  Results do not depend on it. */
morea_status morea_set_launch(morea_problem *p, int32_t blocks_per_sm, int32_t chunk);
morea_status morea_batch_set_launch(morea_batch *b, int32_t blocks_per_sm, int32_t chunk);

/* ---- surrogate pre-screen (a learned model; not part of the paper) ---- */

/* Surrogate input of n_req candidate solutions: per vertex the displacement
 * target - source (voxel units, snapped coordinates, [n_req][V][3] FP32,
 * device) of the solution in slot[r] with the points of request r moved as in
 * morea_eval_partial (chg_off/chg_pts/chg_src/chg_tgt, same layout; an empty
 * request gives the committed solution).  An invalid slot gives NaN features
 * and sets MOREA_DEV_BAD_SLOT. */
morea_status morea_partial_features(morea_problem *p, int32_t n_req, const int32_t *slot,
                                    const int32_t *chg_off, const int32_t *chg_pts, const float *chg_src,
                                    const float *chg_tgt, float *out, void *stream);

typedef struct morea_mlp morea_mlp;                     /* opaque handle */

/* A 3-layer perceptron n_in -> h1 -> h2 -> n_out (ReLU, ReLU, linear) that
 * predicts the (standardised) objectives of a solution from its displacement
 * field, so that only the most promising offspring are evaluated exactly.
 * Weights and activations are BF16 on the tensor cores with FP32
 * accumulation; FP32 master weights and Adam moments are kept.  h1, h2
 * multiples of 64, n_out <= 32, batches up to max_batch.  Parameters start at
 * zero: set them with morea_mlp_set_params. */
morea_status morea_mlp_create(int32_t n_in, int32_t h1, int32_t h2, int32_t n_out, int32_t max_batch,
                              morea_mlp **out);
morea_status morea_mlp_destroy(morea_mlp *n);

/* Number of parameters and the padded input width kin (n_in rounded up to 64).
 * Parameter vector layout (FP32): W1 [h1][kin] (columns >= n_in must be 0),
 * b1 [h1], W2 [h2][h1], b2 [h2], W3 [n_out][h2], b3 [n_out]. */
morea_status morea_mlp_info(const morea_mlp *n, int64_t *n_params, int32_t *padded_inputs);

/* Repair of folded solutions (Sec. 4.3.1), in place, on the stream.
 *
 * src, tgt: device [n_sol][V][3] FP32 coordinates of the two meshes of each
 * solution; updated in place.  noise: device [n_sol][max_points][64][3]
 * standard normal draws (the caller's random numbers).  For each solution:
 * the source mesh, then the target mesh; tets in order and, while a tet is
 * folded, its four vertices in order, each vertex at most once per mesh, at
 * most max_points visits in all.  A visited vertex gets 64 trial positions
 * x + sigma z (rounded to FP32) with sigma = scale times its smallest
 * distance to the plane of a face opposite it in its star (at least
 * 2^-k voxel); the trial with the largest decrease of the star's fold
 * severity is kept (lowest index on ties), and the first vertex without a
 * decreasing trial ends that solution's repair.  fixed: device [V] uint8
 * or NULL; bit a set: axis a of that vertex lies on a face of the image box
 * and keeps its value in every trial.  moved: device [n_sol] number of
 * vertices moved; severity: device [n_sol] fold severity of both meshes
 * afterwards (as morea_check_folds; a degenerate tet is folded but adds no
 * severity, so check the fold flags, not severity 0).  The problem's slots
 * and caches are not touched: evaluate the repaired solutions afterwards.
 * MOREA_EINVAL: null pointers, n_sol < 1, max_points < 1, scale not > 0. */
morea_status morea_repair_folds(morea_problem *p, int32_t n_sol, float *src, float *tgt, const float *noise,
                                int32_t max_points, float scale, const uint8_t *fixed, int32_t *moved,
                                double *severity, void *stream);

/* Objectives of committed slots (a9 from the slots' running totals, which
 * morea_eval_full and morea_commit_partial keep up to date): obj device
 * [n_sol][3], folded device [n_sol], severity device [n_sol] or NULL, as
 * morea_eval_full returns them.  slot: device [n_sol] or NULL (identity).
 * A slot out of range gets NaN objectives and folded = 1.  MOREA_EINVAL:
 * null p/obj/folded, n_sol < 1. */
morea_status morea_slot_objectives(morea_problem *p, int32_t n_sol, const int32_t *slot, double *obj,
                                   uint8_t *folded, double *severity, void *stream);

/* Selection and clustering of MO-RV-GOMEA (Sec. 3).  Host call; needs no
 * GPU.  obj: host [n][3] objectives of the population (finite).  The
 * population is ranked into non-dominated fronts; the ceil(tau n)
 * solutions first in (rank, index) order are selected; objectives are
 * scaled by the selection's range per objective; k leaders are chosen by
 * farthest-first traversal (from the smallest scaled f_0; ties to the
 * lower index); balanced k-means keeps, per cluster, the c = min(|S|,
 * ceil(2 |S| / k)) selected solutions nearest to its mean (ties to the
 * lower index), for at most `iters` rounds or until memberships repeat;
 * every population member is assigned to the nearest mean (ties to the
 * lower cluster).  Squared distances are summed in axis order and nothing
 * is contracted, so results are reproducible bit for bit.
 * Outputs (host): *n_selected and selected [n] (first *n_selected valid);
 * *cluster_size = c and members [k][n] (row q: the c population indices of
 * cluster q, in selection order); pop_cluster [n].  Clusters may overlap.
 * MOREA_EINVAL: n < 1, k < 1, iters < 1, tau not in (0, 1], a non-finite
 * objective, null pointers. */
morea_status morea_cluster(int32_t n, const double *obj, double tau, int32_t k, int32_t iters,
                           int32_t *n_selected, int32_t *selected, int32_t *cluster_size, int32_t *members,
                           int32_t *pop_cluster);

/* Bytes of device workspace morea_sample_elements needs (0 if a count is
 * below 1): one model (12 means + a 12 x 12 factor, FP64) per (cluster,
 * element). */
size_t morea_sample_elements_workspace(int32_t n_clusters, int32_t n_elements);

/* Distributions of the FOS elements per cluster and new partial solutions
 * drawn from them (Sec. 3, optimal mixing).  An element (a, b) has 12
 * variables: source a (x, y, z), source b, target a, target b; variables
 * on a fixed axis of their point keep the parent's value.
 *   src, tgt     device [n_pop][V][3] FP32: the population's coordinates
 *   members      device [n_clusters][cluster_size] population indices
 *   elements     device [n_elements][2] point pairs, 8-byte aligned
 *   fixed        device [V] uint8 axis bits, or NULL
 *   cmult        device [n_clusters] distribution multipliers
 *   req_sol, req_cluster, req_element  device [n_req]: parent, cluster and
 *                element of each new partial solution
 *   z            device [n_req][12] standard normal draws (the caller's)
 *   work         device workspace of morea_sample_elements_workspace()
 *                bytes, 16-byte aligned (caller-owned, not preserved
 *                between calls)
 *   new_src, new_tgt  device [n_req][2][3]: the new coordinates of points a
 *                and b of each request: the candidate rows of a
 *                morea_eval_partial request whose changed points are (a, b)
 * Per (cluster, element): mu = the members' mean (summed in member order),
 * Sigma = the maximum-likelihood covariance, L = the Cholesky factor of
 * Sigma + 1e-6 I over the free variables, all FP64; a request draws
 * mu + cmult L z, rounded to FP32.  An index out of range yields NaN rows.
 * Stream-ordered, no allocation.  MOREA_EINVAL: null pointers, counts out of
 * range, misaligned elements or work, work_bytes too small. */
morea_status morea_sample_elements(morea_problem *p, int32_t n_pop, const float *src, const float *tgt,
                                   int32_t n_clusters, int32_t cluster_size, const int32_t *members,
                                   int32_t n_elements, const int32_t *elements, const uint8_t *fixed,
                                   const float *cmult, int32_t n_req, const int32_t *req_sol,
                                   const int32_t *req_cluster, const int32_t *req_element, const float *z,
                                   void *work, size_t work_bytes, float *new_src, float *new_tgt, void *stream);

/* Initialisation noise for a diverse initial population (Sec. 4.2.2,
 * App. A.5): Gaussian kernels on both images attract the mesh points in
 * rounds while the mesh stays unfolded.
 *   src, tgt  device [n_sol][V][3] FP32, in: the start meshes (e.g. copies
 *             of the reference mesh), out: the result
 *   fixed     device [V] uint8 or NULL; bit a set: axis a of that point does
 *             not move (points on the faces of the image box)
 *   kernels   device [n_sol][2][n_kernels][5] FP32 (cx, cy, cz, sigma, a) for
 *             the source (0) and target (1) mesh of each solution: the
 *             caller's random draws, centres in voxel units, sigma > 0
 *   rounds    device [n_sol][2] int32: the rounds kept for each mesh
 * A round moves every point x to x + sum_k a_k exp(-|c_k - x|^2 /
 * (2 sigma_k^2)) (c_k - x), computed in FP64 over k in order with each
 * operation rounded once, and rounded to FP32; the round is kept if no tet
 * of the moved mesh is folded (exact orientation of the snapped
 * coordinates) and the first round that folds ends the process, so the
 * result is never folded.  At most max_rounds rounds.  Points are not
 * clamped (the snap clamps them at evaluation); with sum_k a_k <= 1 they
 * stay inside the convex hull of the start mesh and the centres.
 * MOREA_EINVAL: null pointers, n_sol < 1, n_kernels < 0, max_rounds < 0,
 * or more than 200 KiB of shared memory (5 n_kernels + 6 V floats). */
morea_status morea_init_noise(morea_problem *p, int32_t n_sol, float *src, float *tgt, const uint8_t *fixed,
                              int32_t n_kernels, const float *kernels, int32_t max_rounds, int32_t *rounds,
                              void *stream);

/* Linkage model and parallel groups of the partial evaluations (Sec. 4.2.1).
 * Host call; needs no GPU.  tets: host [n_tets][4] topology.  The FOS
 * elements are mesh edges chosen by a greedy set cover of the points (the
 * first edge in sorted (a < b) order among those covering the most
 * uncovered points); two elements interact when the tets containing their
 * points overlap; DSATUR colours the interaction graph (most distinct
 * neighbour colours, then largest degree, then lowest index; smallest free
 * colour).  Outputs (host): elements [n_elements][2] point pairs in the
 * order the cover takes them, group [n_elements] colours in
 * [0, n_groups).  Elements of one group touch disjoint tets, so one
 * morea_eval_partial call may carry a request for each of them on the same
 * slot.  MOREA_EINVAL: bad sizes or ids, a point in no tet, or more than
 * max_elements elements. */
morea_status morea_parallel_groups(int32_t n_points, int32_t n_tets, const int32_t *tets, int32_t max_elements,
                                   int32_t *elements, int32_t *group, int32_t *n_elements, int32_t *n_groups);

/* Displacement field of one solution and the label overlap it implies (the
 * evaluation of Sec. 5; not part of the objectives).
 *
 * src, tgt: device [V][3] FP32 coordinates of the solution's two meshes.
 * side 0: for every voxel centre p of the source image inside an unfolded
 * source copy (the exact association of morea_eval_full), dvf(p) = T(p) - p
 * (the forward field); side 1: the same on the target image with T'.
 * dvf: device [nz][ny][nx][3] FP32, or NULL; voxels in no copy are NaN.
 * labels_own / labels_other: device [nz][ny][nx] uint8 label images of
 * this side and of the other side, or both NULL; with them, overlap: device
 * int64 [n_labels][3] = per label l the number of covered voxels with own
 * label l, with label l at the voxel of the other image nearest to T(p)
 * (round half to even, clamped), and with both (Dice = 2 c2 / (c0 + c1)).
 * n_labels <= 64; labels >= n_labels are not counted.  A voxel inside
 * several copies (only with folded or overlapping meshes) is written by one
 * of them and counted once per copy.  MOREA_EINVAL: null p/src/tgt, side
 * not 0/1, labels without overlap or n_labels out of range. */
morea_status morea_displacement(morea_problem *p, const float *src, const float *tgt, int32_t side, float *dvf,
                                const uint8_t *labels_own, const uint8_t *labels_other, int32_t n_labels,
                                int64_t *overlap, void *stream);

/* Warped label image of one solution (the evaluation of Sec. 5).  For every
 * voxel centre p of image `side` inside an unfolded copy of that side's mesh
 * (the association of morea_displacement), warped(p) = labels_other at the
 * voxel of the other image nearest to T(p) (round half to even, clamped);
 * MOREA_NO_LABEL where no copy covers p.  src, tgt: device [V][3] FP32;
 * labels_other, warped: device [nz][ny][nx] uint8 (caller-owned).  Compare
 * warped with this side's own labels (morea_surface_distance) to score the
 * registration.  MOREA_EINVAL: null pointers, side not 0/1. */
#define MOREA_NO_LABEL 255
morea_status morea_warp_labels(morea_problem *p, const float *src, const float *tgt, int32_t side,
                               const uint8_t *labels_other, uint8_t *warped, void *stream);

/* Bytes of device workspace morea_surface_distance needs for an
 * nx x ny x nz image (0 if a size is out of range). */
size_t morea_surface_distance_workspace(int32_t nx, int32_t ny, int32_t nz);

/* Hausdorff distance and its 95th percentile between the surfaces of label
 * `label` in two label images (the evaluation metrics of Sec. 5).
 *   a, b     device [nz][ny][nx] uint8 label images; 1 <= nx, ny, nz <= 1024
 *   label    0..255; a mask is the set of voxels equal to it
 *   work     device workspace of morea_surface_distance_workspace() bytes,
 *            256-byte aligned (caller-owned; its contents need not be
 *            preserved between calls)
 *   out      device double[4]: HD, HD95 (voxel units), |S_a|, |S_b|
 * The surface of a mask is its voxels with a face neighbour outside the
 * mask (beyond the image border counts as outside).  The directed distances
 * of S_a are the Euclidean distances from each of its voxel centres to the
 * nearest voxel centre of S_b (exact: squared distances are integers), and
 * likewise for S_b.  HD is the largest directed distance; HD95 the larger of
 * the two directed 95th percentiles, each by nearest rank (the
 * ceil(0.95 n)-th smallest).  An empty surface gives NaN for HD and HD95.
 * Stream-ordered, no allocation, no host synchronisation.  MOREA_EINVAL:
 * sizes out of range, null pointers, work_bytes too small or work not
 * 256-byte aligned. */
morea_status morea_surface_distance(int32_t nx, int32_t ny, int32_t nz, const uint8_t *a, const uint8_t *b,
                                    int32_t label, void *work, size_t work_bytes, double *out, void *stream);

/* Read and clear the network's device status word (synchronises the
 * stream).  Bit 0 (MOREA_DEV_MLP_WAIT_TIMEOUT): a wait inside a
 * tensor-core product gave up (its outputs are invalid).  No counterpart in
 * the paper; the bounded waits are the kernels' own safeguard. */
#define MOREA_DEV_MLP_WAIT_TIMEOUT 1u
morea_status morea_mlp_device_status(morea_mlp *n, uint32_t *bits, void *stream);

/* Copy the parameter vector in (resets the Adam state) / out.  host or device. */
morea_status morea_mlp_set_params(morea_mlp *n, const float *params, void *stream);
morea_status morea_mlp_get_params(morea_mlp *n, float *params, void *stream);

/* y [batch][n_out] = network(x [batch][n_in]) (device FP32). */
morea_status morea_mlp_forward(morea_mlp *n, int32_t batch, const float *x, float *y, void *stream);

/* Gradient of the mean squared error between network(x) and t
 * ([batch][n_out]) w.r.t. the parameter vector (grads, device FP32, may be
 * NULL) and the loss (device scalar, may be NULL); no update. */
morea_status morea_mlp_gradients(morea_mlp *n, int32_t batch, const float *x, const float *t, float *grads,
                                 float *loss, void *stream);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on the mean squared error of
 * (x, t) with learning rate lr; loss (device scalar, may be NULL) is the loss
 * before the step. */
morea_status morea_mlp_train_step(morea_mlp *n, int32_t batch, const float *x, const float *t, float lr,
                                  float *loss, void *stream);

/* Instrumentation for benchmarks (not a step of the method; the paper has no
 * counterpart).  flags bit 0: record a CUDA event pair on the call's stream
 * around every launch of the rasterisation/sampling kernel (the hot loop);
 * bit 1: after each such launch, count the voxel visits it made (one extra
 * small kernel, outside the event pair).  flags = 0 turns both off.  Every
 * call resets the accumulated figures.  Creates CUDA events on first use; no
 * device memory is allocated. */
morea_status morea_profile(morea_problem *p, uint32_t flags);

/* Synchronise the events recorded since the last morea_profile call and
 * return the summed kernel time in ms, the number of timed launches and the
 * counted voxel visits (any output may be NULL). */
morea_status morea_profile_read(morea_problem *p, double *raster_ms, int64_t *launches,
                                int64_t *visits);

/* Largest n_sol * n_tets that morea_fold_magnitude_noalloc accepts (its
 * fixed scratch holds one 16-byte record per (solution, tet): 8 MiB). */
#define MOREA_NOALLOC_MAX_TET_EVALS 524288

/* Fold constraint and deformation magnitude of n_sol solutions without a
 * problem handle and without allocating any memory.  The paper has no
 * counterpart to this entry point; it exists for callers that cannot call
 * cudaMalloc -- code running inside another allocator or memory pool that
 * must not re-enter it, or environments that only hand out pre-sized buffers
 * -- and so cannot create a problem handle either.
 *   tets        device [n_tets][4] vertex ids in [0, n_points) (any
 *               orientation: a tet whose reference volume is negative is
 *               re-ordered, as at problem creation).  A tet with an id out of
 *               range, or with a zero reference volume (which problem
 *               creation rejects), is not evaluated: every solution gets
 *               f_mag = NaN and folded = 1.
 *   ref_points  device [n_points][3] initial mesh (gives the reference signs)
 *   cdelta      device [n_tets] elasticity factor of each tet
 *   nx, ny, nz, subvoxel_bits   image box and snapping grid, chosen exactly
 *               as morea_create_problem chooses them: subvoxel_bits 0 takes
 *               the largest k <= 8 with max(nx, ny, nz) 2^k <= 65536 and
 *               4 n_tets nx ny nz 8^k < 2^63 (the exact 64-bit severity
 *               sum); a given k that breaks either bound returns
 *               MOREA_EINVAL
 *   src_pts, tgt_pts  device [n_sol][n_points][3]
 *   f_mag       device [n_sol] out: f_magnitude (obj[1] of morea_eval_full)
 *   folded      device [n_sol] out; severity device [n_sol] out or NULL
 * The per-(solution, tet) intermediates go to one fixed device array inside
 * the library (8 MiB, held by every GPU that loads the library until the
 * process exits).  n_sol * n_tets above MOREA_NOALLOC_MAX_TET_EVALS returns
 * MOREA_EINVAL before anything is launched.  All calls on a device share
 * that array: calls whose work overlaps on the GPU (on unordered streams)
 * race and give wrong results; calls on one stream are safe.  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * The address is kept for the life of the process, so the entry point is not
 * supported on a device after cudaDeviceReset of that device.
 * Nothing is allocated and no memory of the caller is kept. */
morea_status morea_fold_magnitude_noalloc(int32_t n_sol, int32_t n_points, int32_t n_tets,
                                          const int32_t *tets, const float *ref_points,
                                          const float *cdelta, int32_t nx, int32_t ny, int32_t nz,
                                          int32_t subvoxel_bits, const float *src_pts,
                                          const float *tgt_pts, double *f_mag, uint8_t *folded,
                                          double *severity, void *stream);

/* Static description of a status code. */
const char *morea_status_string(morea_status s);

#ifdef __cplusplus
}
#endif

#endif /* MOREA_H */
