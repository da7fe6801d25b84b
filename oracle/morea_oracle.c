/*
 * MOREA objective oracle: a plain, slow, FP64/int64 CPU restatement of the
 * objectives and the fold constraint of MOREA (Andreadis, Bosman,
 * Alderliesten, GECCO 2023, arXiv 2303.04873).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke check
 * and the benchmark's CPU-baseline leg may load or execute this code.  The
 * product path (the CUDA kernels behind libmorea) never calls it, and the two
 * share no source: no headers, helpers, tables or constants.
 *
 * Everything is written as the plain definition: explicit loops over every
 * voxel centre of every tetrahedron's bounding box, an exact inside test per
 * (voxel, tet) pair, a barycentric map, an 8-corner weighted sum for the
 * trilinear sample, sums in tet order.  No incremental evaluation, no
 * blocking, no reordering.
 *
 * Paper passages followed (section / equation):
 *   deformation magnitude  Sec. 4.1.1, f_magnitude equation; App. A.1
 *   image intensity        Sec. 4.1.2, f_intensity and h equations; App. A.2
 *   guidance               Sec. 4.1.3, f_guidance and g equations; App. A.3
 *   fold constraint        Sec. 4.1.4; App. A.4 (signed-volume sign flips)
 *   partial evaluation     Sec. 1 and Sec. 4.2.1 (re-evaluate dependent tets)
 *
 * Readings where the paper is silent (shared with the CUDA path by
 * specification, not by code):
 *   R1 snap: coordinates are clamped to the image box [-0.5, n-0.5] and
 *      rounded half-to-even onto a grid of 2^-k voxel (k = subvoxel_bits);
 *      q = rint((x + 0.5) * 2^k), so voxel centre i sits at (i + 1/2) 2^k.
 *   R2 orientation: orient(a,b,c,d) = (b-a).((c-a)x(d-a)) over the integers;
 *      tets with a negative reference volume are re-ordered (swap of the last
 *      two vertices) so every reference sign is +; a zero reference volume is
 *      an error.  A copy is folded iff its orient value is <= 0 (App. A.4:
 *      a fold flips the sign; zero counts as folded).
 *   R3 voxel association: a voxel centre belongs to a tet iff it lies inside
 *      the tet after the symbolic perturbation p + (e, e^2, e^3), e -> 0+
 *      (simulation of simplicity).  On a conforming, box-filling, unfolded
 *      mesh every voxel centre is then counted exactly once (the defect the
 *      paper attributes to the prior voxel association in App. A.2).
 *      A folded copy is not rasterised (it contributes no voxels).
 *   R4 trilinear sampling clamps the position to [0, n-1] per axis and uses
 *      the cell i0 = min(floor(y), n-2).
 *   R5 spoke edges are the four centroid-to-vertex segments.
 *   R6 severity = sum over folded copies (both meshes) of |orient| / (6 2^3k)
 *      (the absolute signed volume in voxel^3).
 *   R7 guidance distance maps are exact Euclidean distances from voxel
 *      centres to the group's contour points; mapped positions sample the
 *      other side's map trilinearly.  Group weights |C^k|/|G| multiply as in
 *      the printed formula.
 *   R8 pair-transfer guidance (the prior, exact measure of App. A.3): mean of
 *      |T(g_s) - g_t|^2 and |T'(g_t) - g_s|^2 over located points; a point
 *      is located with R3 on its snapped coordinates.
 *   R9 h in the foreground/background mode jumps at b = 0 (from (a-b)^2 to
 *      1).  The case is decided on the sample b of the stored image values
 *      at the exact T(p), as Sec. 4.1.2 defines h on the sampled
 *      intensities: T(p) of a voxel centre is kept as an exact rational, so
 *      the clamp, the cell and a zero fraction are exact, and b is the
 *      8-corner sum with each fraction rounded once (FP64).  Where a caller evaluates T(p) and b in lower
 *      precision the decision can differ close to b = 0; orc_set_perturbation
 *      turns on a per-voxel report of exactly those voxels (see below).
 *   R13 sampled estimator (App. A.2, the paper's own estimator; estimator =
 *      1).  Per tet copy with orient D > 0: N = floor(rate * vol + 1/2)
 *      points (capped at 2^24), vol = D / (6 2^3k) voxel^3 in FP64, rate the
 *      given float.  Point j = 0 .. N-1 takes the 4-D Sobol point of
 *      Gray-code index j (Joe-Kuo direction numbers; natural index
 *      j ^ (j >> 1)), each 32-bit coordinate XOR-ed with a digital shift
 *      derived from the copy's coordinates: FNV-1a (64-bit) over the copy's
 *      12 snapped coordinates as little-endian int32 words, vertex by vertex,
 *      then shift_d = high 32 bits of the (d+1)-th splitmix64 output from
 *      that state.  u_d = (x_d + 1/2) 2^-32, e_d = -log u_d, lambda_d =
 *      e_d / sum e (uniform on the tet), p = sum lambda_d v_d on the own
 *      copy and T(p) = sum lambda_d w_d on the other (voxel units); both
 *      images are sampled trilinearly (R4), and h, the guidance term (own
 *      map sampled at p) and the counts (N per copy) enter as in the voxel
 *      estimator.  Only h_mode PLAIN_SSD.
 *   R14 repair (Sec. 4.3.1).  Source mesh first, then target mesh; within a
 *      mesh the tets are visited in order and, if folded at that moment,
 *      their four vertices in order, each vertex at most once per mesh.  A
 *      vertex v at float position x gets sigma = scale * (the smallest
 *      distance, over the tets of its star, from v to the plane of the face
 *      opposite v), at least 1/2^k voxel; trial k (k = 0..63) is
 *      x + sigma z_k rounded to float, z_k the caller's standard normal
 *      draws for this (solution, visit, trial).  The trial with the largest
 *      strictly positive decrease of the star's severity (sum of |orient|
 *      over its folded tets; ties to the lowest k) replaces x; if no trial
 *      decreases it, the repair of the solution stops.  At most max_points
 *      visits per solution.  FP64 without contraction, so the float trial
 *      positions are the same on every machine.  With fixed axes given (bit
 *      a of fixed[v]: axis a of point v lies on a face of the image box and
 *      stays there), a trial keeps those coordinates of x.
 *   R15 displacement field and label overlap (the evaluation of Sec. 5):
 *      for every voxel centre p of one image inside an unfolded copy (R3),
 *      dvf(p) = T(p) - p with the FP64 barycentric map; voxels in no copy
 *      are NaN, and a voxel inside several copies (folded or overlapping
 *      meshes only) takes the first copy in tet order.  Label overlap: the
 *      nearest voxel of the other image to the exact (rational) T(p), round
 *      half to even, clamped to the image, gives the pulled-back label; per label l
 *      the counts of covered voxels with own label l, with pulled-back
 *      label l, and with both.  The warped label image holds the
 *      pulled-back label per voxel, 255 in no copy.
 *   R18 initialisation noise (Sec. 4.2.2, App. A.5: Gaussian kernels
 *      on both images attract the mesh points, in rounds, as long as no
 *      fold appears).  Per mesh, kernels (c_k, sigma_k, a_k) are the
 *      caller's draws; a round moves x by sum_k a_k g_k(x) (c_k - x) with
 *      g_k(x) = exp(-|c_k - x|^2 / (2 sigma_k^2)), in FP64 over k in order,
 *      rounded to float, with fixed axes kept; it is kept if the moved
 *      mesh has no folded tet, and the first folding round ends the
 *      process.  exp is the function gexp below (range reduction by ln 2
 *      and a Taylor series, every operation one rounded IEEE operation), so
 *      positions are reproducible bit for bit.
 *
 * Perturbation report (test support, off by default).  R9 and R15 turn a
 * real number into a decision (the sign of b; the nearest voxel of T(p)).
 * A kernel that evaluates T(p) = t0 + M (p - s0) and the trilinear sample
 * in FP32 gets the same decision unless the exact value lies within its
 * rounding error of the threshold.  Given a relative radius gamma_pos for
 * the position and gamma_val for the sample, the oracle bounds per voxel
 *   eps_a = gamma_pos (|t0_a| + sum_b |M_ab| |p_b - s0_b| + 1)
 * (M the exact linear part of the map, s0, t0 vertex 0 of the two copies)
 * and, over the cells the box y +- eps touches,
 *   tau = sum_a L_a eps_a + gamma_val V
 * (L_a the largest |difference| along axis a of neighbouring stored
 * values, V the largest |stored value|): every position within eps and
 * every sample within tau of the exact ones.  A voxel is ambiguous when the
 * decision is not constant over that range; its record counts it, with the
 * spread of h it allows (R9) or the candidate labels (R15).  The report
 * never changes a returned value.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

#define ORC_MAX_GROUPS 8
#define ORC_MAX_SAMPLES (1LL << 24)

typedef struct { int64_t x, y, z; } orc_i3;

typedef struct {
    int32_t nx, ny, nz, pad0;
    const double *img_s;            /* [nz][ny][nx] stored values, as double */
    const double *img_t;
    int32_t n_points, n_tets;
    const int32_t *tets;            /* [T][4] */
    const float *ref_points;        /* [V][3] */
    const int32_t *tet_label;       /* [T] or NULL */
    const double *tissue_factor;    /* [L] or NULL */
    int32_t n_labels;
    int32_t n_guid;
    const float *guid_s;            /* [n_guid][3] */
    const float *guid_t;
    const int32_t *guid_group;      /* [n_guid] or NULL */
    double trunc_radius;            /* <= 0: 2.5% of nx */
    int32_t h_mode, g_mode, subvoxel_bits, estimator;   /* estimator: 0 voxels (R3), 1 samples (R13) */
    double sampling_rate;           /* R13: points per voxel^3 (the float value given) */
    const uint8_t *tissue_mask;     /* [nz][ny][nx] tissue label per voxel of I_s, or NULL (App. A.1) */
} orc_problem;

typedef struct {
    double e_img[2];
    double e_guid[2];
    int64_t n_vox[2];
    int64_t n_gp[2];
    double e_mag;
    uint64_t sev;
    int32_t folded;                 /* bit 0: source copy, bit 1: target copy */
    int32_t pad;
    int64_t amb_n[2];               /* perturbation report: ambiguous voxels (R9) */
    double amb_slack[2];            /* and the spread of h they allow */
} orc_tet;

typedef struct {
    double obj[3];                  /* f_intensity, f_magnitude, f_guidance */
    double severity;
    double s_img, s_guid, s_mag;
    int64_t n_vox, n_gp, n_folded;
    uint64_t sev_raw;
    int32_t folded, pad;
} orc_result;

typedef struct {
    orc_problem p;
    int32_t *tets;                  /* positively oriented */
    double *cdelta;                 /* elasticity factor per tet */
    int G;
    double wgt[ORC_MAX_GROUPS];
    double r;
    double *dist[2];                /* [G][N] maps of the source / target contours */
    int64_t S;                      /* 2^k */
    double amb_pos, amb_val;        /* perturbation report radii (0: off) */
} orc_state;

/* ------------------------------------------------------------------ */
/* R1: snap a coordinate onto the 2^-k voxel grid                      */
/* ------------------------------------------------------------------ */
static int64_t snap1(float xf, int n, int k)
{
    double x = (double)xf;
    x = fmax(x, -0.5);
    x = fmin(x, (double)n - 0.5);
    return (int64_t)rint((x + 0.5) * ldexp(1.0, k));
}

static orc_i3 snap3(const orc_state *st, const float *pt)
{
    orc_i3 q;
    q.x = snap1(pt[0], st->p.nx, st->p.subvoxel_bits);
    q.y = snap1(pt[1], st->p.ny, st->p.subvoxel_bits);
    q.z = snap1(pt[2], st->p.nz, st->p.subvoxel_bits);
    return q;
}

/* R2: integer orientation determinant (six times the signed volume). */
static int64_t orient(orc_i3 a, orc_i3 b, orc_i3 c, orc_i3 d)
{
    int64_t bx = b.x - a.x, by = b.y - a.y, bz = b.z - a.z;
    int64_t cx = c.x - a.x, cy = c.y - a.y, cz = c.z - a.z;
    int64_t dx = d.x - a.x, dy = d.y - a.y, dz = d.z - a.z;
    return bx * (cy * dz - cz * dy) + by * (cz * dx - cx * dz) + bz * (cx * dy - cy * dx);
}

static int64_t orient_arr(const orc_i3 v[4])
{
    return orient(v[0], v[1], v[2], v[3]);
}

/* D_i(p): orientation with vertex i replaced by p. */
static int64_t face_value(const orc_i3 v[4], int i, orc_i3 p)
{
    orc_i3 w[4];
    memcpy(w, v, sizeof(w));
    w[i] = p;
    return orient_arr(w);
}

/* R3: is p inside the positively oriented tet v after the symbolic
 * perturbation (e, e^2, e^3)?  D_i is affine in p, so
 * D_i(p + (e, e^2, e^3)) = D_i(p) + g_x e + g_y e^2 + g_z e^3 and its sign
 * for e -> 0+ is the first nonzero of (D_i(p), g_x, g_y, g_z). */
static int inside_sos(const orc_i3 v[4], orc_i3 p)
{
    for (int i = 0; i < 4; ++i) {
        int64_t d = face_value(v, i, p);
        if (d > 0) continue;
        if (d < 0) return 0;
        orc_i3 px = p, py = p, pz = p;
        px.x += 1; py.y += 1; pz.z += 1;
        int64_t gx = face_value(v, i, px) - d;
        int64_t gy = face_value(v, i, py) - d;
        int64_t gz = face_value(v, i, pz) - d;
        int s = gx != 0 ? (gx > 0) : gy != 0 ? (gy > 0) : (gz > 0);
        if (!s) return 0;
    }
    return 1;
}

/* R4: trilinear sample as the weighted sum of the 8 corners of cell i0
 * with fractions f. */
static double trilinear_cell(const double *img, int nx, int ny, const int i0[3], const double f[3])
{
    double v = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                size_t idx = ((size_t)(i0[2] + dz) * ny + (size_t)(i0[1] + dy)) * nx + (size_t)(i0[0] + dx);
                v += w * img[idx];
            }
    return v;
}

/* R4 at a position y given in FP64: clamp to [0, n-1], cell
 * i0 = min(floor(y), n - 2), fraction y - i0. */
static double trilinear(const double *img, int nx, int ny, int nz, const double y[3])
{
    int n[3] = {nx, ny, nz};
    int i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double c = fmin(fmax(y[a], 0.0), (double)(n[a] - 1));
        int i = (int)floor(c);
        if (i > n[a] - 2) i = n[a] - 2;
        i0[a] = i;
        f[a] = c - (double)i;
    }
    return trilinear_cell(img, nx, ny, i0, f);
}

/* Exact rationals for the voxel-centre map (128-bit integers; gcc and
 * clang provide them on every 64-bit target). */
__extension__ typedef __int128 orc_i128;

static orc_i128 floor_div128(orc_i128 a, orc_i128 b)   /* b > 0 */
{
    orc_i128 q = a / b;
    if (a % b != 0 && a < 0) --q;
    return q;
}

/* R4 at the exact position num[a] / den (den > 0): the clamp, the cell
 * and whether a fraction is 0 or 1 are decided exactly; each fraction is
 * then rounded once.  A position on a voxel centre samples that voxel's
 * stored value exactly. */
static double trilinear_exact(const double *img, int nx, int ny, int nz, const orc_i128 num[3], orc_i128 den)
{
    int n[3] = {nx, ny, nz};
    int i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        orc_i128 c = num[a] < 0 ? 0 : num[a];
        orc_i128 top = (orc_i128)(n[a] - 1) * den;
        if (c > top) c = top;
        orc_i128 q = c / den;
        if (q > n[a] - 2) q = n[a] - 2;
        i0[a] = (int)q;
        f[a] = (double)(c - q * den) / (double)den;
    }
    return trilinear_cell(img, nx, ny, i0, f);
}

/* h of Sec. 4.1.2: mode 0 = squared difference; mode 1 = the printed case
 * split on foreground (> 0) and background (== 0) intensities (R9). */
static double h_fn(int mode, double a, double b)
{
    if (mode == 0) return (a - b) * (a - b);
    if (a > 0.0 && b > 0.0) return (a - b) * (a - b);
    if (a == 0.0 && b == 0.0) return 0.0;
    return 1.0;
}

/* ------------------------------------------------------------------ */
/* Perturbation report (test support; see the header)                 */
/* ------------------------------------------------------------------ */

static orc_i3 orc_add(orc_i3 p, int a)
{
    if (a == 0) p.x += 1; else if (a == 1) p.y += 1; else p.z += 1;
    return p;
}

/* eps[a]: the radius of position a of the map at voxel centre p.  A row
 * of the map whose exact entries M_ab are all in {-1, 0, 1} is evaluated
 * exactly in FP32 (the products and sums of 2^-k-grid values below 2^10
 * need at most 18 bits), so its radius is 0. */
static void map_radius(const orc_state *st, const orc_i3 own[4], int64_t D, const orc_i3 oth[4], orc_i3 p,
                       double eps[3])
{
    double S = (double)st->S;
    int64_t g[4][3];                           /* d D_i / d p_b per snapped unit (integers) */
    for (int i = 0; i < 4; ++i) {
        int64_t d0 = face_value(own, i, p);
        for (int b = 0; b < 3; ++b) g[i][b] = face_value(own, i, orc_add(p, b)) - d0;
    }
    double s0[3] = {(double)own[0].x / S - 0.5, (double)own[0].y / S - 0.5, (double)own[0].z / S - 0.5};
    double pv[3] = {(double)p.x / S - 0.5, (double)p.y / S - 0.5, (double)p.z / S - 0.5};
    for (int a = 0; a < 3; ++a) {
        double t0 = (a == 0 ? oth[0].x : a == 1 ? oth[0].y : oth[0].z) / S - 0.5;
        double acc = fabs(t0) + 1.0;
        int unit_row = 1;
        for (int b = 0; b < 3; ++b) {
            /* M_ab = sum_i q_i,a g_i,b / D exactly (the -1/2 offsets cancel: sum_i g_i = 0) */
            orc_i128 num = 0;
            for (int i = 0; i < 4; ++i) {
                int64_t q = a == 0 ? oth[i].x : a == 1 ? oth[i].y : oth[i].z;
                num += (orc_i128)q * g[i][b];
            }
            if (!(num == 0 || num == D || num == -(orc_i128)D)) unit_row = 0;
            acc += fabs((double)num / (double)D) * fabs(pv[b] - s0[b]);
        }
        eps[a] = unit_row ? 0.0 : st->amb_pos * acc;
    }
}

/* tau: the radius of the trilinear sample of img over the positions within
 * eps of y (R4 clamping and cells).  fix[a] >= 0 marks an axis whose
 * clamped position is the grid index fix[a] in every evaluation within eps
 * (see exact_axes).  On such an axis the fraction is 0 (fix[a] <= n - 2) or
 * 1 (fix[a] = n - 1, cell n - 2): the corner fix[a] carries the whole
 * weight.  With fraction 0 an FP32 lerp returns that corner exactly; with
 * fraction 1 it reads the other corner too, which then counts for the
 * rounding part.  If every corner that can carry weight is 0, the exact
 * sample is 0 and so is every FP32 evaluation within eps (a lerp of zeros
 * is 0, and fmaf(1, 0 - v, v) is 0): the radius is 0. */
static double value_radius(const orc_state *st, const double *img, const double y[3], const double eps[3],
                           const int fix[3])
{
    const orc_problem *P = &st->p;
    int n[3] = {P->nx, P->ny, P->nz};
    int r0[3], r1[3], w0[3], w1[3];          /* corners read (rounding) and corners with weight */
    for (int a = 0; a < 3; ++a) {
        if (fix[a] >= 0) {
            w0[a] = w1[a] = fix[a];
            r0[a] = fix[a] == n[a] - 1 ? n[a] - 2 : fix[a];
            r1[a] = fix[a];
            continue;
        }
        double lo = fmin(fmax(y[a] - eps[a], 0.0), (double)(n[a] - 1));
        double hi = fmin(fmax(y[a] + eps[a], 0.0), (double)(n[a] - 1));
        int c0 = (int)floor(lo), c1 = (int)floor(hi);
        if (c0 > n[a] - 2) c0 = n[a] - 2;
        if (c1 > n[a] - 2) c1 = n[a] - 2;
        r0[a] = w0[a] = c0;
        r1[a] = w1[a] = c1 + 1;
    }
    double V = 0.0, L[3] = {0.0, 0.0, 0.0};
    int weighted_nonzero = 0;
    for (int k = r0[2]; k <= r1[2]; ++k)
        for (int j = r0[1]; j <= r1[1]; ++j)
            for (int i = r0[0]; i <= r1[0]; ++i) {
                size_t idx = ((size_t)k * P->ny + (size_t)j) * P->nx + (size_t)i;
                double v = img[idx];
                if (fabs(v) > V) V = fabs(v);
                if (v != 0.0 && i >= w0[0] && i <= w1[0] && j >= w0[1] && j <= w1[1] && k >= w0[2] && k <= w1[2])
                    weighted_nonzero = 1;
                if (fix[0] < 0 && i < r1[0]) L[0] = fmax(L[0], fabs(img[idx + 1] - v));
                if (fix[1] < 0 && j < r1[1]) L[1] = fmax(L[1], fabs(img[idx + (size_t)P->nx] - v));
                if (fix[2] < 0 && k < r1[2]) L[2] = fmax(L[2], fabs(img[idx + (size_t)P->nx * P->ny] - v));
            }
    double tau = 0.0;
    for (int a = 0; a < 3; ++a)
        if (fix[a] < 0) tau += L[a] * eps[a];
    return weighted_nonzero ? tau + st->amb_val * V : 0.0;
}

/* fix[a] of value_radius: the grid index at which the clamped position
 * sits in every evaluation within eps -- an exact integer with eps[a] = 0,
 * or a range that clamps as a whole to 0 or to n - 1 -- else -1. */
static void exact_axes(const orc_i128 num[3], orc_i128 den, const int n[3], const double y[3], const double eps[3],
                       int fix[3])
{
    for (int a = 0; a < 3; ++a) {
        fix[a] = -1;
        if (y[a] + eps[a] <= 0.0) { fix[a] = 0; continue; }
        if (y[a] - eps[a] >= (double)(n[a] - 1)) { fix[a] = n[a] - 1; continue; }
        if (eps[a] != 0.0) continue;
        orc_i128 c = num[a] < 0 ? 0 : num[a];
        orc_i128 top = (orc_i128)(n[a] - 1) * den;
        if (c > top) c = top;
        if (c % den == 0) fix[a] = (int)(c / den);
    }
}

/* R9 report: the spread of h when the case is decided on any b' within tau
 * of b (the compared value stays b). */
static double h_spread(double a, double b, double tau)
{
    int pos = b + tau > 0.0, zero = b - tau <= 0.0 && b + tau >= 0.0, neg = b - tau < 0.0;
    double lo = INFINITY, hi = -INFINITY, v;
#define ORC_CASE(c, val) if (c) { v = (val); lo = fmin(lo, v); hi = fmax(hi, v); }
    if (a > 0.0) {
        ORC_CASE(pos, (a - b) * (a - b));
        ORC_CASE(zero || neg, 1.0);
    } else if (a == 0.0) {
        ORC_CASE(zero, 0.0);
        ORC_CASE(pos || neg, 1.0);
    } else {
        ORC_CASE(1, 1.0);
    }
#undef ORC_CASE
    return hi - lo;
}

static int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

static int64_t ceil_div(int64_t a, int64_t b)
{
    return -floor_div(-a, b);
}

/* Barycentric map of Sec. 4.2.1's dual-dynamic model: the point p of the
 * own copy, with lambda_i = D_i(p) / D, goes to sum_i lambda_i * w_i where
 * w_i are the other copy's vertices in voxel units. */
static void bary_map(const orc_state *st, const orc_i3 own[4], int64_t D, const orc_i3 oth[4],
                     orc_i3 p, double y[3])
{
    double S = (double)st->S;
    y[0] = y[1] = y[2] = 0.0;
    for (int i = 0; i < 4; ++i) {
        double lam = (double)face_value(own, i, p) / (double)D;
        y[0] += lam * ((double)oth[i].x / S - 0.5);
        y[1] += lam * ((double)oth[i].y / S - 0.5);
        y[2] += lam * ((double)oth[i].z / S - 0.5);
    }
}

/* The same map at a voxel centre p as an exact rational per axis,
 * y_a = num[a] / den with den > 0: the other copy's vertices are
 * w_i = q_i / S - 1/2 and sum_i D_i(p) = D, so
 * y = (2 sum_i D_i(p) q_i - D S) / (2 D S). */
static orc_i128 bary_exact(const orc_state *st, const orc_i3 own[4], int64_t D, const orc_i3 oth[4], orc_i3 p,
                           orc_i128 num[3])
{
    orc_i128 sx = 0, sy = 0, sz = 0;
    for (int i = 0; i < 4; ++i) {
        orc_i128 di = face_value(own, i, p);
        sx += di * oth[i].x;
        sy += di * oth[i].y;
        sz += di * oth[i].z;
    }
    orc_i128 DS = (orc_i128)D * st->S;
    num[0] = 2 * sx - DS;
    num[1] = 2 * sy - DS;
    num[2] = 2 * sz - DS;
    return 2 * DS;
}

/* R15: the voxel index nearest to num / den on an axis of n voxels, round
 * half to even, clamped to the image; decided exactly. */
static int64_t nearest_exact(orc_i128 num, orc_i128 den, int n)
{
    orc_i128 t = 2 * num + den, d2 = 2 * den;          /* y + 1/2 = t / d2 */
    orc_i128 m = floor_div128(t, d2);
    if (m * d2 == t && (m & 1)) m -= 1;                /* tie: y = m - 1/2, take the even neighbour */
    if (m < 0) m = 0;
    if (m > n - 1) m = n - 1;
    return (int64_t)m;
}

/* One side of one tet: side 0 samples source voxels in the source copy and
 * compares with the target image at T(p); side 1 is the symmetric term with
 * T' (the two sums of f_intensity and the two g terms of f_guidance). */
static void eval_side_sampled(const orc_state *st, const orc_i3 own[4], const orc_i3 oth[4], int side,
                              orc_tet *rec);

static void eval_side(const orc_state *st, const orc_i3 own[4], const orc_i3 oth[4], int side,
                      orc_tet *rec)
{
    const orc_problem *P = &st->p;
    int64_t D = orient_arr(own);
    if (D <= 0) return;                                /* R3: folded copy not rasterised */
    int sampled = P->estimator == 1;
    const double *img_own = side == 0 ? P->img_s : P->img_t;
    const double *img_oth = side == 0 ? P->img_t : P->img_s;
    int64_t S = st->S, H = st->S / 2;
    int n[3] = {P->nx, P->ny, P->nz};
    int64_t lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        int64_t mn = INT64_MAX, mx = INT64_MIN;
        for (int i = 0; i < 4; ++i) {
            int64_t c = a == 0 ? own[i].x : a == 1 ? own[i].y : own[i].z;
            if (c < mn) mn = c;
            if (c > mx) mx = c;
        }
        lo[a] = ceil_div(mn - H, S);
        hi[a] = floor_div(mx - H, S);
        if (lo[a] < 0) lo[a] = 0;
        if (hi[a] > n[a] - 1) hi[a] = n[a] - 1;
    }
    double e_img = 0.0, e_guid = 0.0;
    int64_t nv = 0;
    if (!sampled)                                     /* R3 voxel sums; R13 sums below */
    for (int64_t k = lo[2]; k <= hi[2]; ++k)
        for (int64_t j = lo[1]; j <= hi[1]; ++j)
            for (int64_t i = lo[0]; i <= hi[0]; ++i) {
                orc_i3 p = {i * S + H, j * S + H, k * S + H};
                if (!inside_sos(own, p)) continue;
                orc_i128 num[3];
                orc_i128 den = bary_exact(st, own, D, oth, p, num);
                double y[3] = {(double)num[0] / (double)den, (double)num[1] / (double)den,
                               (double)num[2] / (double)den};
                size_t idx = ((size_t)k * P->ny + (size_t)j) * P->nx + (size_t)i;
                double a = img_own[idx];
                double b = trilinear_exact(img_oth, P->nx, P->ny, P->nz, num, den);
                e_img += h_fn(P->h_mode, a, b);
                nv += 1;
                if (P->h_mode == 1 && st->amb_pos > 0.0) {     /* perturbation report (R9) */
                    double eps[3];
                    int fix[3];
                    map_radius(st, own, D, oth, p, eps);
                    exact_axes(num, den, n, y, eps, fix);
                    double tau = value_radius(st, img_oth, y, eps, fix);
                    if (tau > 0.0 && fabs(b) <= tau) {
                        rec->amb_n[side] += 1;
                        rec->amb_slack[side] += h_spread(a, b, tau);
                    }
                }
                if (P->g_mode == 0) {
                    for (int g = 0; g < st->G; ++g) {
                        double dg = st->dist[side][(size_t)g * ((size_t)P->nx * P->ny * P->nz) + idx];
                        if (dg < st->r) {
                            double dm = trilinear(st->dist[1 - side] + (size_t)g * ((size_t)P->nx * P->ny * P->nz),
                                                  P->nx, P->ny, P->nz, y);
                            e_guid += st->wgt[g] * (st->r - dg) / st->r * (dg - dm) * (dg - dm);
                        }
                    }
                }
            }
    int64_t ngp = 0;
    if (P->g_mode == 1) {
        for (int m = 0; m < P->n_guid; ++m) {
            const float *gown = side == 0 ? P->guid_s + 3 * m : P->guid_t + 3 * m;
            const float *goth = side == 0 ? P->guid_t + 3 * m : P->guid_s + 3 * m;
            orc_i3 p = snap3(st, gown);
            if (!inside_sos(own, p)) continue;
            double y[3];
            bary_map(st, own, D, oth, p, y);
            double ex = y[0] - (double)goth[0], ey = y[1] - (double)goth[1], ez = y[2] - (double)goth[2];
            e_guid += ex * ex + ey * ey + ez * ez;
            ngp += 1;
        }
    }
    rec->e_img[side] = e_img;
    rec->e_guid[side] = e_guid;
    rec->n_vox[side] = nv;
    rec->n_gp[side] = ngp;
    if (sampled) eval_side_sampled(st, own, oth, side, rec);   /* R13 replaces the voxel sums */
}

/* ------------------------------------------------------------------ */
/* R13: the sampled estimator of App. A.2                              */
/* ------------------------------------------------------------------ */

/* Sobol direction numbers V[d][b] (32-bit) of the first four dimensions:
 * d = 0 is the van der Corput sequence; d = 1, 2, 3 use the primitive
 * polynomials x + 1, x^2 + x + 1, x^3 + x + 1 (degree s, inner coefficients
 * a) with initial numbers m = {1}, {1, 3}, {1, 3, 1} (Joe and Kuo's table),
 * continued by m_k = m_{k-s} ^ (m_{k-s} << s) ^ sum_i a_i (m_{k-i} << i). */
static uint32_t sobol_v[4][32];
static int sobol_ready = 0;

static void sobol_init(void)
{
    if (sobol_ready) return;
    static const int deg[4] = {0, 1, 2, 3};
    static const int poly[4] = {0, 0, 1, 1};
    static const uint32_t m0[4][3] = {{0, 0, 0}, {1, 0, 0}, {1, 3, 0}, {1, 3, 1}};
    for (int b = 0; b < 32; ++b) sobol_v[0][b] = 1u << (31 - b);
    for (int d = 1; d < 4; ++d) {
        int s = deg[d];
        uint32_t m[33];
        for (int k = 1; k <= s; ++k) m[k] = m0[d][k - 1];
        for (int k = s + 1; k <= 32; ++k) {
            uint32_t v = m[k - s] ^ (m[k - s] << s);
            for (int i = 1; i < s; ++i)
                if ((poly[d] >> (s - 1 - i)) & 1) v ^= m[k - i] << i;
            m[k] = v;
        }
        for (int k = 1; k <= 32; ++k) sobol_v[d][k - 1] = m[k] << (32 - k);
    }
    sobol_ready = 1;
}

/* Coordinate d of the Sobol point with Gray-code index j (unshifted). */
static uint32_t sobol_gray(uint64_t j, int d)
{
    uint64_t n = j ^ (j >> 1);
    uint32_t x = 0;
    for (int b = 0; n != 0 && b < 32; ++b, n >>= 1)
        if (n & 1) x ^= sobol_v[d][b];
    return x;
}

static uint64_t fnv1a64(const uint8_t *p, size_t n)
{
    uint64_t h = 0xcbf29ce484222325ULL;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 0x100000001b3ULL;
    }
    return h;
}

/* splitmix64: advance the state by the golden-ratio increment, then mix. */
static uint64_t splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Digital shifts of one tet copy, from its snapped coordinates. */
static void copy_shifts(const orc_i3 v[4], uint32_t shift[4])
{
    uint8_t bytes[48];
    for (int i = 0; i < 4; ++i) {
        int64_t c[3] = {v[i].x, v[i].y, v[i].z};
        for (int a = 0; a < 3; ++a) {
            uint32_t w = (uint32_t)(int32_t)c[a];
            for (int q = 0; q < 4; ++q) bytes[12 * i + 4 * a + q] = (uint8_t)(w >> (8 * q));
        }
    }
    uint64_t state = fnv1a64(bytes, sizeof(bytes));
    for (int d = 0; d < 4; ++d) shift[d] = (uint32_t)(splitmix64_next(&state) >> 32);
}

/* Barycentric coordinates of sample j of a copy with the given shifts. */
static void sample_lambda(const uint32_t shift[4], uint64_t j, double lam[4])
{
    double e[4], sum = 0.0;
    for (int d = 0; d < 4; ++d) {
        uint32_t x = sobol_gray(j, d) ^ shift[d];
        double u = ((double)x + 0.5) / 4294967296.0;
        e[d] = -log(u);
        sum += e[d];
    }
    for (int d = 0; d < 4; ++d) lam[d] = e[d] / sum;
}

static int64_t sample_count(const orc_state *st, int64_t D)
{
    double S = (double)st->S;
    double vol = (double)D / (6.0 * S * S * S);
    int64_t n = (int64_t)floor(st->p.sampling_rate * vol + 0.5);
    return n > ORC_MAX_SAMPLES ? ORC_MAX_SAMPLES : n;
}

static void eval_side_sampled(const orc_state *st, const orc_i3 own[4], const orc_i3 oth[4], int side,
                              orc_tet *rec)
{
    const orc_problem *P = &st->p;
    int64_t D = orient_arr(own);
    if (D <= 0) return;                                /* folded copy: no samples */
    const double *img_own = side == 0 ? P->img_s : P->img_t;
    const double *img_oth = side == 0 ? P->img_t : P->img_s;
    size_t N3 = (size_t)P->nx * P->ny * P->nz;
    double S = (double)st->S;
    double vo[4][3], vt[4][3];
    for (int i = 0; i < 4; ++i) {
        vo[i][0] = (double)own[i].x / S - 0.5; vo[i][1] = (double)own[i].y / S - 0.5; vo[i][2] = (double)own[i].z / S - 0.5;
        vt[i][0] = (double)oth[i].x / S - 0.5; vt[i][1] = (double)oth[i].y / S - 0.5; vt[i][2] = (double)oth[i].z / S - 0.5;
    }
    uint32_t shift[4];
    copy_shifts(own, shift);
    int64_t n = sample_count(st, D);
    double e_img = 0.0, e_guid = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double lam[4], p[3] = {0, 0, 0}, y[3] = {0, 0, 0};
        sample_lambda(shift, (uint64_t)j, lam);
        for (int i = 0; i < 4; ++i)
            for (int a = 0; a < 3; ++a) {
                p[a] += lam[i] * vo[i][a];
                y[a] += lam[i] * vt[i][a];
            }
        double a = trilinear(img_own, P->nx, P->ny, P->nz, p);
        double b = trilinear(img_oth, P->nx, P->ny, P->nz, y);
        e_img += h_fn(P->h_mode, a, b);
        if (P->g_mode == 0) {
            for (int g = 0; g < st->G; ++g) {
                double dg = trilinear(st->dist[side] + (size_t)g * N3, P->nx, P->ny, P->nz, p);
                if (dg < st->r) {
                    double dm = trilinear(st->dist[1 - side] + (size_t)g * N3, P->nx, P->ny, P->nz, y);
                    e_guid += st->wgt[g] * (st->r - dg) / st->r * (dg - dm) * (dg - dm);
                }
            }
        }
    }
    rec->e_img[side] = e_img;
    rec->e_guid[side] += e_guid;
    rec->n_vox[side] = n;
}

static double len3(double x, double y, double z)
{
    return sqrt(x * x + y * y + z * z);
}

/* Per-tet summands of every objective and of the fold constraint. */
void orc_eval_tet(const orc_state *st, const float *src, const float *tgt, int t, orc_tet *rec)
{
    memset(rec, 0, sizeof(*rec));
    orc_i3 qs[4], qt[4];
    for (int i = 0; i < 4; ++i) {
        int v = st->tets[4 * t + i];
        qs[i] = snap3(st, src + 3 * (size_t)v);
        qt[i] = snap3(st, tgt + 3 * (size_t)v);
    }
    /* Sec. 4.1.4 / App. A.4: sign flip against the (positive) reference sign */
    int64_t Ds = orient_arr(qs), Dt = orient_arr(qt);
    if (Ds <= 0) { rec->folded |= 1; rec->sev += (uint64_t)(Ds < 0 ? -Ds : Ds); }
    if (Dt <= 0) { rec->folded |= 2; rec->sev += (uint64_t)(Dt < 0 ? -Dt : Dt); }
    /* Sec. 4.1.1: 6 edges + 4 spokes (R5), c_delta (ls - lt)^2 */
    double S = (double)st->S;
    double e = 0.0;
    for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b) {
            double ls = len3((qs[b].x - qs[a].x) / S, (qs[b].y - qs[a].y) / S, (qs[b].z - qs[a].z) / S);
            double lt = len3((qt[b].x - qt[a].x) / S, (qt[b].y - qt[a].y) / S, (qt[b].z - qt[a].z) / S);
            e += (ls - lt) * (ls - lt);
        }
    double cs[3] = {0, 0, 0}, ct[3] = {0, 0, 0};
    for (int i = 0; i < 4; ++i) {
        cs[0] += qs[i].x / 4.0; cs[1] += qs[i].y / 4.0; cs[2] += qs[i].z / 4.0;
        ct[0] += qt[i].x / 4.0; ct[1] += qt[i].y / 4.0; ct[2] += qt[i].z / 4.0;
    }
    for (int i = 0; i < 4; ++i) {
        double ls = len3((qs[i].x - cs[0]) / S, (qs[i].y - cs[1]) / S, (qs[i].z - cs[2]) / S);
        double lt = len3((qt[i].x - ct[0]) / S, (qt[i].y - ct[1]) / S, (qt[i].z - ct[2]) / S);
        e += (ls - lt) * (ls - lt);
    }
    rec->e_mag = st->cdelta[t] * e;
    /* Sec. 4.1.2 / 4.1.3: both sampling sides */
    eval_side(st, qs, qt, 0, rec);
    eval_side(st, qt, qs, 1, rec);
}

static void finish(const orc_state *st, orc_result *res)
{
    const orc_problem *P = &st->p;
    res->obj[0] = res->n_vox > 0 ? res->s_img / (double)res->n_vox : 0.0;
    res->obj[1] = res->s_mag / (10.0 * (double)P->n_tets);
    if (P->g_mode == 0)
        res->obj[2] = res->n_vox > 0 ? res->s_guid / (double)res->n_vox : 0.0;
    else if (P->g_mode == 1)
        res->obj[2] = res->n_gp > 0 ? res->s_guid / (double)res->n_gp : 0.0;
    else
        res->obj[2] = 0.0;
    res->folded = res->n_folded > 0;
    double S = (double)st->S;
    res->severity = (double)res->sev_raw / (6.0 * S * S * S);
}

static void add_rec(orc_result *res, const orc_tet *r, double sign)
{
    res->s_img += sign * (r->e_img[0] + r->e_img[1]);
    res->s_guid += sign * (r->e_guid[0] + r->e_guid[1]);
    res->s_mag += sign * r->e_mag;
    int64_t is = sign > 0 ? 1 : -1;
    res->n_vox += is * (r->n_vox[0] + r->n_vox[1]);
    res->n_gp += is * (r->n_gp[0] + r->n_gp[1]);
    res->n_folded += is * (int64_t)(((r->folded & 1) != 0) + ((r->folded & 2) != 0));
    if (sign > 0) res->sev_raw += r->sev; else res->sev_raw -= r->sev;
}

/* Totals of f_intensity, f_magnitude, f_guidance (sums in tet order). */
void orc_totals(const orc_state *st, const orc_tet *recs, orc_result *res)
{
    memset(res, 0, sizeof(*res));
    for (int t = 0; t < st->p.n_tets; ++t) add_rec(res, &recs[t], 1.0);
    finish(st, res);
}

/* Full evaluation of one solution (src, tgt: [V][3]). recs may be NULL. */
int orc_eval(const orc_state *st, const float *src, const float *tgt, orc_tet *recs, orc_result *res)
{
    orc_tet *own = recs;
    if (!own) {
        own = (orc_tet *)malloc(sizeof(orc_tet) * (size_t)st->p.n_tets);
        if (!own) return ORC_ENOMEM;
    }
    for (int t = 0; t < st->p.n_tets; ++t) orc_eval_tet(st, src, tgt, t, &own[t]);
    orc_totals(st, own, res);
    if (!recs) free(own);
    return ORC_OK;
}

/* Partial evaluation (Sec. 1, Sec. 4.2.1): only the tets with a changed
 * vertex are re-evaluated; result = old totals + sum(new - old). */
int orc_eval_partial(const orc_state *st, const float *old_src, const float *old_tgt,
                     const float *new_src, const float *new_tgt, int n_chg, const int32_t *chg,
                     const orc_result *old_tot, orc_result *res, int32_t *n_affected)
{
    const orc_problem *P = &st->p;
    char *mark = (char *)calloc((size_t)P->n_points, 1);
    if (!mark) return ORC_ENOMEM;
    for (int m = 0; m < n_chg; ++m) {
        if (chg[m] < 0 || chg[m] >= P->n_points) { free(mark); return ORC_EINVAL; }
        mark[chg[m]] = 1;
    }
    *res = *old_tot;
    int32_t na = 0;
    for (int t = 0; t < P->n_tets; ++t) {
        const int32_t *tv = st->tets + 4 * t;
        if (!(mark[tv[0]] || mark[tv[1]] || mark[tv[2]] || mark[tv[3]])) continue;
        orc_tet ro, rn;
        orc_eval_tet(st, old_src, old_tgt, t, &ro);
        orc_eval_tet(st, new_src, new_tgt, t, &rn);
        add_rec(res, &ro, -1.0);
        add_rec(res, &rn, 1.0);
        ++na;
    }
    free(mark);
    finish(st, res);
    if (n_affected) *n_affected = na;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* set-up                                                              */
/* ------------------------------------------------------------------ */

void orc_free(orc_state *st)
{
    if (!st) return;
    free(st->tets);
    free(st->cdelta);
    free(st->dist[0]);
    free(st->dist[1]);
    free(st);
}

/* App. A.1, elasticity from tissue overlap: c = sum_k frac_k f_k +
 * (1 - sum_k frac_k) f_0 with label 0 the background.  frac_k is taken on
 * the voxel grid: the voxel centres of the tet's (positively oriented)
 * reference copy by the association of R3, counted per label of the mask;
 * then c = sum_l count_l f_l / sum_l count_l, in label order.  A tet with
 * no voxel centre keeps the factor of its label. */
static void tissue_factor_of(orc_state *st, int t)
{
    const orc_problem *P = &st->p;
    int64_t count[64];
    memset(count, 0, sizeof(count));
    orc_i3 v[4];
    for (int i = 0; i < 4; ++i) v[i] = snap3(st, P->ref_points + 3 * (size_t)st->tets[4 * t + i]);
    int64_t S = st->S, H = st->S / 2;
    int n[3] = {P->nx, P->ny, P->nz};
    int64_t lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        int64_t mn = INT64_MAX, mx = INT64_MIN;
        for (int i = 0; i < 4; ++i) {
            int64_t c = a == 0 ? v[i].x : a == 1 ? v[i].y : v[i].z;
            if (c < mn) mn = c;
            if (c > mx) mx = c;
        }
        lo[a] = ceil_div(mn - H, S);
        hi[a] = floor_div(mx - H, S);
        if (lo[a] < 0) lo[a] = 0;
        if (hi[a] > n[a] - 1) hi[a] = n[a] - 1;
    }
    for (int64_t k = lo[2]; k <= hi[2]; ++k)
        for (int64_t j = lo[1]; j <= hi[1]; ++j)
            for (int64_t i = lo[0]; i <= hi[0]; ++i) {
                orc_i3 p = {i * S + H, j * S + H, k * S + H};
                if (!inside_sos(v, p)) continue;
                count[P->tissue_mask[((size_t)k * P->ny + (size_t)j) * P->nx + (size_t)i]] += 1;
            }
    int64_t total = 0;
    double s = 0.0;
    for (int l = 0; l < P->n_labels; ++l) {
        total += count[l];
        s += (double)count[l] * P->tissue_factor[l];
    }
    if (total > 0) st->cdelta[t] = s / (double)total;
}

/* R7: brute-force Euclidean distance map of one contour point set. */
static void distance_map(const orc_problem *P, const float *pts, int g, double *out)
{
    for (int k = 0; k < P->nz; ++k)
        for (int j = 0; j < P->ny; ++j)
            for (int i = 0; i < P->nx; ++i) {
                double best = INFINITY;
                for (int m = 0; m < P->n_guid; ++m) {
                    int gm = P->guid_group ? P->guid_group[m] : 0;
                    if (gm != g) continue;
                    double d = len3(i - (double)pts[3 * m], j - (double)pts[3 * m + 1], k - (double)pts[3 * m + 2]);
                    if (d < best) best = d;
                }
                out[((size_t)k * P->ny + j) * P->nx + i] = best;
            }
}

int orc_setup(const orc_problem *P, orc_state **out)
{
    *out = NULL;
    if (P->nx < 2 || P->ny < 2 || P->nz < 2) return ORC_EINVAL;
    if (P->subvoxel_bits < 2 || P->subvoxel_bits > 14) return ORC_EINVAL;
    int64_t S = (int64_t)1 << P->subvoxel_bits;
    int nmax = P->nx > P->ny ? P->nx : P->ny;
    if (P->nz > nmax) nmax = P->nz;
    if ((int64_t)nmax * S > ((int64_t)1 << 16)) return ORC_EINVAL;
    if (P->n_points < 4 || P->n_tets < 1 || !P->tets || !P->ref_points) return ORC_EINVAL;
    if (P->h_mode < 0 || P->h_mode > 1 || P->g_mode < 0 || P->g_mode > 2) return ORC_EINVAL;
    if (P->estimator < 0 || P->estimator > 1) return ORC_EINVAL;
    if (P->estimator == 1 && (P->h_mode != 0 || !(P->sampling_rate > 0.0))) return ORC_EINVAL;
    sobol_init();
    if (P->n_guid < 0 || (P->n_guid > 0 && (!P->guid_s || !P->guid_t))) return ORC_EINVAL;
    orc_state *st = (orc_state *)calloc(1, sizeof(orc_state));
    if (!st) return ORC_ENOMEM;
    st->p = *P;
    st->S = S;
    st->tets = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)P->n_tets);
    st->cdelta = (double *)malloc(sizeof(double) * (size_t)P->n_tets);
    if (!st->tets || !st->cdelta) { orc_free(st); return ORC_ENOMEM; }
    /* R2: positive reference orientation */
    for (int t = 0; t < P->n_tets; ++t) {
        orc_i3 q[4];
        for (int i = 0; i < 4; ++i) {
            int v = P->tets[4 * t + i];
            if (v < 0 || v >= P->n_points) { orc_free(st); return ORC_EINVAL; }
            st->tets[4 * t + i] = v;
            q[i] = snap3(st, P->ref_points + 3 * (size_t)v);
        }
        int64_t D = orient_arr(q);
        if (D == 0) { orc_free(st); return ORC_EINVAL; }
        if (D < 0) {
            int32_t tmp = st->tets[4 * t + 2];
            st->tets[4 * t + 2] = st->tets[4 * t + 3];
            st->tets[4 * t + 3] = tmp;
        }
        /* App. A.1: per-tet elasticity factor from its tissue label */
        int lab = P->tet_label ? P->tet_label[t] : 0;
        if (P->tissue_factor) {
            if (lab < 0 || lab >= P->n_labels) { orc_free(st); return ORC_EINVAL; }
            st->cdelta[t] = P->tissue_factor[lab];
        } else {
            st->cdelta[t] = 1.0;
        }
    }
    if (P->tissue_mask) {
        if (!P->tissue_factor || P->n_labels > 64) { orc_free(st); return ORC_EINVAL; }
        size_t N = (size_t)P->nx * P->ny * P->nz;
        for (size_t v = 0; v < N; ++v)
            if (P->tissue_mask[v] >= P->n_labels) { orc_free(st); return ORC_EINVAL; }
        for (int t = 0; t < P->n_tets; ++t) tissue_factor_of(st, t);
    }
    /* guidance groups, weights |C^k| / |G| and truncation radius */
    st->G = 0;
    for (int m = 0; m < P->n_guid; ++m) {
        int g = P->guid_group ? P->guid_group[m] : 0;
        if (g < 0 || g >= ORC_MAX_GROUPS) { orc_free(st); return ORC_EINVAL; }
        if (g + 1 > st->G) st->G = g + 1;
    }
    for (int g = 0; g < st->G; ++g) {
        int cnt = 0;
        for (int m = 0; m < P->n_guid; ++m) cnt += (P->guid_group ? P->guid_group[m] : 0) == g;
        st->wgt[g] = (double)cnt / (double)P->n_guid;
    }
    st->r = P->trunc_radius > 0.0 ? P->trunc_radius : 0.025 * (double)P->nx;
    if (P->g_mode == 0 && st->G > 0) {
        size_t N = (size_t)P->nx * P->ny * P->nz;
        for (int s = 0; s < 2; ++s) {
            st->dist[s] = (double *)malloc(sizeof(double) * N * (size_t)st->G);
            if (!st->dist[s]) { orc_free(st); return ORC_ENOMEM; }
            for (int g = 0; g < st->G; ++g)
                distance_map(P, s == 0 ? P->guid_s : P->guid_t, g, st->dist[s] + (size_t)g * N);
        }
    }
    *out = st;
    return ORC_OK;
}

/* Turn the perturbation report on (radii > 0) or off (0). */
void orc_set_perturbation(orc_state *st, double gamma_pos, double gamma_val)
{
    st->amb_pos = gamma_pos > 0.0 ? gamma_pos : 0.0;
    st->amb_val = gamma_val > 0.0 ? gamma_val : 0.0;
}

/* accessors used by the tests */
int orc_n_groups(const orc_state *st) { return st->G; }
double orc_radius(const orc_state *st) { return st->r; }
const int32_t *orc_oriented_tets(const orc_state *st) { return st->tets; }
const double *orc_cdelta(const orc_state *st) { return st->cdelta; }
const double *orc_distance(const orc_state *st, int side, int g)
{
    if (!st->dist[side] || g < 0 || g >= st->G) return NULL;
    return st->dist[side] + (size_t)g * ((size_t)st->p.nx * st->p.ny * st->p.nz);
}

/* Exposed building blocks, so the tests can pin them one by one. */
int64_t orc_snap1(float x, int n, int k) { return snap1(x, n, k); }
int64_t orc_orient(const int64_t *a, const int64_t *b, const int64_t *c, const int64_t *d)
{
    orc_i3 A = {a[0], a[1], a[2]}, B = {b[0], b[1], b[2]}, C = {c[0], c[1], c[2]}, D = {d[0], d[1], d[2]};
    return orient(A, B, C, D);
}
int orc_inside(const int64_t *tet12, const int64_t *p3)
{
    orc_i3 v[4];
    for (int i = 0; i < 4; ++i) { v[i].x = tet12[3 * i]; v[i].y = tet12[3 * i + 1]; v[i].z = tet12[3 * i + 2]; }
    orc_i3 p = {p3[0], p3[1], p3[2]};
    return inside_sos(v, p);
}
double orc_trilinear(const double *img, int nx, int ny, int nz, const double *y)
{
    return trilinear(img, nx, ny, nz, y);
}
double orc_h(int mode, double a, double b) { return h_fn(mode, a, b); }

/* R13 building blocks */
uint32_t orc_sobol(uint64_t j, int d) { sobol_init(); return (d >= 0 && d < 4) ? sobol_gray(j, d) : 0; }
uint64_t orc_fnv1a64(const uint8_t *p, size_t n) { return fnv1a64(p, n); }
uint64_t orc_splitmix64(uint64_t *state) { return splitmix64_next(state); }
void orc_copy_shifts(const int64_t *tet12, uint32_t *shift)
{
    orc_i3 v[4];
    for (int i = 0; i < 4; ++i) { v[i].x = tet12[3 * i]; v[i].y = tet12[3 * i + 1]; v[i].z = tet12[3 * i + 2]; }
    copy_shifts(v, shift);
}
void orc_sample_lambda(const uint32_t *shift, uint64_t j, double *lam) { sobol_init(); sample_lambda(shift, j, lam); }

/* ------------------------------------------------------------------ */
/* R14: repair of folded solutions (Sec. 4.3.1)                        */
/* ------------------------------------------------------------------ */

static orc_i3 vertex_at(const orc_state *st, const float *X, int v) { return snap3(st, X + 3 * (size_t)v); }

/* sum of |orient| over the folded tets of v's star, v placed at q */
static uint64_t star_severity(const orc_state *st, const float *X, int v, orc_i3 q)
{
    uint64_t sev = 0;
    for (int t = 0; t < st->p.n_tets; ++t) {
        const int32_t *tv = st->tets + 4 * t;
        if (tv[0] != v && tv[1] != v && tv[2] != v && tv[3] != v) continue;
        orc_i3 c[4];
        for (int i = 0; i < 4; ++i) c[i] = tv[i] == v ? q : vertex_at(st, X, tv[i]);
        int64_t D = orient_arr(c);
        if (D <= 0) sev += (uint64_t)(D < 0 ? -D : D);
    }
    return sev;
}

/* distance (voxels) from p to the plane through a, b, c; infinity if degenerate */
static double plane_distance(const orc_state *st, orc_i3 p, orc_i3 a, orc_i3 b, orc_i3 c)
{
    int64_t ux = b.x - a.x, uy = b.y - a.y, uz = b.z - a.z;
    int64_t vx = c.x - a.x, vy = c.y - a.y, vz = c.z - a.z;
    int64_t nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
    double nn = (double)nx * (double)nx + (double)ny * (double)ny + (double)nz * (double)nz;
    if (nn == 0.0) return INFINITY;
    int64_t num = nx * (p.x - a.x) + ny * (p.y - a.y) + nz * (p.z - a.z);
    double d = fabs((double)num) / sqrt(nn);
    return d / (double)st->S;
}

static double repair_sigma(const orc_state *st, const float *X, int v, double scale)
{
    orc_i3 p = vertex_at(st, X, v);
    double dmin = INFINITY;
    for (int t = 0; t < st->p.n_tets; ++t) {
        const int32_t *tv = st->tets + 4 * t;
        orc_i3 f[3];
        int n = 0, has = 0;
        for (int i = 0; i < 4; ++i) {
            if (tv[i] == v) has = 1;
            else if (n < 3) f[n++] = vertex_at(st, X, tv[i]);
        }
        if (!has || n != 3) continue;
        double d = plane_distance(st, p, f[0], f[1], f[2]);
        if (d < dmin) dmin = d;
    }
    double sigma = scale * dmin;
    double floor_s = 1.0 / (double)st->S;
    if (!(sigma >= floor_s)) sigma = floor_s;          /* also when no plane is finite */
    return sigma;
}

static int tet_folded(const orc_state *st, const float *X, int t)
{
    orc_i3 c[4];
    for (int i = 0; i < 4; ++i) c[i] = vertex_at(st, X, st->tets[4 * t + i]);
    return orient_arr(c) <= 0;
}

/* Repair of one solution in place.  noise: [max_points][64][3] standard
 * normal draws.  Returns the number of moved points; *sev_raw = sum of
 * |orient| over the folded copies of both meshes afterwards. */
int orc_repair(const orc_state *st, float *src, float *tgt, const float *noise, int max_points, double scale,
               uint64_t *sev_raw, const uint8_t *fixed)
{
    const orc_problem *P = &st->p;
    int moved = 0, visits = 0, stop = 0;
    char *done = (char *)malloc((size_t)P->n_points);
    if (!done) return -1;
    for (int m = 0; m < 2 && !stop; ++m) {
        float *X = m == 0 ? src : tgt;
        memset(done, 0, (size_t)P->n_points);
        for (int t = 0; t < P->n_tets && !stop; ++t) {
            if (!tet_folded(st, X, t)) continue;
            for (int i = 0; i < 4 && !stop; ++i) {
                int v = st->tets[4 * t + i];
                if (done[v]) continue;
                done[v] = 1;
                if (visits >= max_points) { stop = 1; break; }
                double sigma = repair_sigma(st, X, v, scale);
                uint64_t before = star_severity(st, X, v, vertex_at(st, X, v));
                int64_t best_gain = 0;
                int best_k = -1;
                float best[3] = {0, 0, 0};
                for (int k = 0; k < 64; ++k) {
                    const float *z = noise + ((size_t)visits * 64 + k) * 3;
                    float q[3];
                    for (int a = 0; a < 3; ++a) {
                        if (fixed && ((fixed[v] >> a) & 1)) {      /* a fixed axis keeps its value */
                            q[a] = X[3 * (size_t)v + a];
                            continue;
                        }
                        double step = sigma * (double)z[a];
                        double pos = (double)X[3 * (size_t)v + a] + step;
                        q[a] = (float)pos;
                    }
                    uint64_t after = star_severity(st, X, v, snap3(st, q));
                    int64_t gain = (int64_t)before - (int64_t)after;
                    if (gain > best_gain) {
                        best_gain = gain;
                        best_k = k;
                        best[0] = q[0]; best[1] = q[1]; best[2] = q[2];
                    }
                }
                ++visits;
                if (best_k < 0) { stop = 1; break; }          /* every trial deteriorates: abort */
                for (int a = 0; a < 3; ++a) X[3 * (size_t)v + a] = best[a];
                ++moved;
            }
        }
    }
    free(done);
    uint64_t sev = 0;
    for (int m = 0; m < 2; ++m) {
        const float *X = m == 0 ? src : tgt;
        for (int t = 0; t < P->n_tets; ++t) {
            orc_i3 c[4];
            for (int i = 0; i < 4; ++i) c[i] = vertex_at(st, X, st->tets[4 * t + i]);
            int64_t D = orient_arr(c);
            if (D <= 0) sev += (uint64_t)(D < 0 ? -D : D);
        }
    }
    *sev_raw = sev;
    return moved;
}

double orc_repair_sigma(const orc_state *st, const float *X, int v, double scale)
{
    return repair_sigma(st, X, v, scale);
}

/* ------------------------------------------------------------------ */
/* R15: displacement field and label overlap                           */
/* ------------------------------------------------------------------ */

/* R15: the voxel index nearest to position y on an axis of n voxels
 * (round half to even, clamped to the image). */
static int64_t nearest_index(double y, int n)
{
    double r = rint(y);
    if (!(r >= 0.0)) r = 0.0;
    if (r > (double)(n - 1)) r = (double)(n - 1);
    return (int64_t)r;
}

/* cand (optional, [N][8]): the labels the perturbation report allows per
 * covered voxel (all eight equal the pulled-back label where the nearest
 * voxel is the same over the whole range). */
int orc_dvf(const orc_state *st, const float *src, const float *tgt, int side, double *dvf,
            const uint8_t *lab_own, const uint8_t *lab_oth, int n_labels, int64_t *counts, uint8_t *warped,
            uint8_t *cand)
{
    const orc_problem *P = &st->p;
    const size_t N = (size_t)P->nx * P->ny * P->nz;
    char *covered = (char *)calloc(N, 1);
    if (!covered) return ORC_ENOMEM;
    if (dvf)
        for (size_t q = 0; q < 3 * N; ++q) dvf[q] = NAN;
    if (counts) memset(counts, 0, sizeof(int64_t) * 3 * (size_t)n_labels);
    if (warped) memset(warped, 255, N);                   /* 255: in no copy */
    if (cand) memset(cand, 255, 8 * N);
    const float *Xo = side == 0 ? src : tgt, *Xt = side == 0 ? tgt : src;
    int64_t S = st->S, H = st->S / 2;
    int n[3] = {P->nx, P->ny, P->nz};
    for (int t = 0; t < P->n_tets; ++t) {
        orc_i3 own[4], oth[4];
        for (int i = 0; i < 4; ++i) {
            int v = st->tets[4 * t + i];
            own[i] = snap3(st, Xo + 3 * (size_t)v);
            oth[i] = snap3(st, Xt + 3 * (size_t)v);
        }
        int64_t D = orient_arr(own);
        if (D <= 0) continue;                              /* folded copy: not rasterised */
        int64_t lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            int64_t mn = INT64_MAX, mx = INT64_MIN;
            for (int i = 0; i < 4; ++i) {
                int64_t c = a == 0 ? own[i].x : a == 1 ? own[i].y : own[i].z;
                if (c < mn) mn = c;
                if (c > mx) mx = c;
            }
            lo[a] = ceil_div(mn - H, S);
            hi[a] = floor_div(mx - H, S);
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > n[a] - 1) hi[a] = n[a] - 1;
        }
        for (int64_t k = lo[2]; k <= hi[2]; ++k)
            for (int64_t j = lo[1]; j <= hi[1]; ++j)
                for (int64_t i = lo[0]; i <= hi[0]; ++i) {
                    orc_i3 p = {i * S + H, j * S + H, k * S + H};
                    if (!inside_sos(own, p)) continue;
                    size_t idx = ((size_t)k * P->ny + (size_t)j) * P->nx + (size_t)i;
                    if (covered[idx]) continue;
                    covered[idx] = 1;
                    orc_i128 num[3];
                    orc_i128 den = bary_exact(st, own, D, oth, p, num);
                    double y[3] = {(double)num[0] / (double)den, (double)num[1] / (double)den,
                                   (double)num[2] / (double)den};
                    if (dvf) {
                        dvf[3 * idx] = y[0] - (double)i;
                        dvf[3 * idx + 1] = y[1] - (double)j;
                        dvf[3 * idx + 2] = y[2] - (double)k;
                    }
                    if (counts || warped) {
                        int64_t m[3];
                        for (int a = 0; a < 3; ++a) m[a] = nearest_exact(num[a], den, n[a]);
                        size_t jdx = ((size_t)m[2] * P->ny + (size_t)m[1]) * P->nx + (size_t)m[0];
                        int lb = lab_oth[jdx];
                        if (warped) warped[idx] = (uint8_t)lb;
                        if (cand) {                           /* perturbation report (R15) */
                            int64_t c[3][2];
                            double eps[3] = {0.0, 0.0, 0.0};
                            if (st->amb_pos > 0.0) map_radius(st, own, D, oth, p, eps);
                            for (int a = 0; a < 3; ++a) {
                                c[a][0] = nearest_index(y[a] - eps[a], n[a]);
                                c[a][1] = nearest_index(y[a] + eps[a], n[a]);
                            }
                            for (int q = 0; q < 8; ++q) {
                                size_t cdx = ((size_t)c[2][(q >> 2) & 1] * P->ny + (size_t)c[1][(q >> 1) & 1]) * P->nx +
                                             (size_t)c[0][q & 1];
                                cand[8 * idx + q] = lab_oth[cdx];
                            }
                        }
                        if (!counts) continue;
                        int la = lab_own[idx];
                        if (la < n_labels) counts[3 * la] += 1;
                        if (lb < n_labels) counts[3 * lb + 1] += 1;
                        if (la == lb && la < n_labels) counts[3 * la + 2] += 1;
                    }
                }
    }
    free(covered);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* R18: initialisation noise by Gaussian attraction kernels            */
/* ------------------------------------------------------------------ */

/* exp(t) for t <= 0 (R18): t = n ln2 + r with n = rint(t / ln2), exp(r) by
 * its Taylor series to degree 13 in Horner form (s <- 1 + r s / k for
 * k = 13 .. 1; the truncation is below 1e-17 relative for |r| <= ln2 / 2),
 * then scaled by 2^n exactly.  Zero below -64.  Every operation is a single
 * rounded IEEE operation (this file is compiled without contraction). */
static double gexp(double t)
{
    const double LN2 = 0.6931471805599453;
    if (!(t >= -64.0)) return 0.0;
    double n = rint(t / LN2);
    double r = t - n * LN2;
    double s = 1.0;
    for (int k = 13; k >= 1; --k) s = 1.0 + (r * s) / (double)k;
    return ldexp(s, (int)n);
}

double orc_gexp(double t) { return gexp(t); }

static int mesh_folded(const orc_state *st, const float *X)
{
    for (int t = 0; t < st->p.n_tets; ++t)
        if (tet_folded(st, X, t)) return 1;
    return 0;
}

/* One mesh X [V][3] (in/out) under K kernels [K][5] = (cx, cy, cz, sigma,
 * a): a round moves every point x to x + sum_k a_k exp(-|c_k - x|^2 /
 * (2 sigma_k^2)) (c_k - x), in FP64 over k in order, rounded to float;
 * coordinates whose bit is set in fixed[v] (bit a = axis a) stay.  The
 * round is kept if no tet of the moved mesh is folded (R2 on the snapped
 * coordinates); the first round that folds ends the process.  Returns the
 * number of kept rounds (<= max_rounds). */
int orc_init_noise(const orc_state *st, float *X, const float *kernels, int K, const uint8_t *fixed, int max_rounds)
{
    const int V = st->p.n_points;
    float *Y = (float *)malloc(sizeof(float) * 3 * (size_t)V);
    if (!Y) return -1;
    int kept = 0;
    for (int round = 0; round < max_rounds; ++round) {
        for (int v = 0; v < V; ++v) {
            double x[3] = {X[3 * v], X[3 * v + 1], X[3 * v + 2]};
            double d[3] = {0.0, 0.0, 0.0};
            for (int k = 0; k < K; ++k) {
                const float *c = kernels + 5 * k;
                double dx = (double)c[0] - x[0], dy = (double)c[1] - x[1], dz = (double)c[2] - x[2];
                double q = (dx * dx + dy * dy) + dz * dz;
                double sig = c[3];
                double w = (double)c[4] * gexp(-(q / (2.0 * (sig * sig))));
                d[0] = d[0] + w * dx;
                d[1] = d[1] + w * dy;
                d[2] = d[2] + w * dz;
            }
            for (int a = 0; a < 3; ++a)
                Y[3 * v + a] = (fixed && (fixed[v] >> a) & 1) ? X[3 * v + a] : (float)(x[a] + d[a]);
        }
        if (mesh_folded(st, Y)) break;
        memcpy(X, Y, sizeof(float) * 3 * (size_t)V);
        ++kept;
    }
    free(Y);
    return kept;
}
