// Surface distances between two label masks: the Hausdorff distance and its
// 95th percentile, the evaluation metrics of Sec. 5 (reading R17), behind
// morea_surface_distance.  Every step is exact integer arithmetic:
//
//   k_surface    per voxel, bit 0 = on the surface of mask a, bit 1 = of
//                mask b (a mask voxel with a face neighbour outside the mask
//                or beyond the border); the two surface sizes and the box
//                bounding both surfaces.  Every surface voxel lies in the
//                box, so the transforms below are exact inside it when
//                computed from the box alone: the later passes skip the
//                rest of the image
//   k_edt_x      squared distance along x to the nearest surface voxel of
//                the same row, for both surfaces (one warp per row; ballots
//                find the nearest set position on either side)
//   k_edt_line   f'(j) = min_q f(q) + (j - q)^2 along y, then along z: after
//                the three 1-D passes f is the exact squared Euclidean
//                distance to the nearest surface voxel (the separable
//                decomposition of the squared distance, Saito and Toriwaki
//                1994); columns of 32 x-neighbours are staged in shared
//                memory, so the loads are coalesced and the minimisation
//                reads shared memory only
//   k_directed   at every surface voxel of a, the squared distance to b's
//                surface (b's transform), and vice versa: maximum and a
//                histogram of squared distances per direction; the last
//                block to finish takes the nearest-rank 95th percentile of
//                each direction from its histogram (chunked block scan) and
//                writes the outputs
//
// Workspace: surface bits [N] u8, four int32 fields [N], two histograms of
// (nx-1)^2 + (ny-1)^2 + (nz-1)^2 + 1 bins, counters.  Nothing is allocated.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include <cuda_runtime.h>

#include "../../include/morea.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kInf = 1 << 29;              // "no surface voxel"; above any real squared distance
constexpr int kMaxExtent = 1024;
constexpr int kLineThreadsY = 8;

struct Counters {
    unsigned long long n[2];                 // |S_a|, |S_b|
    unsigned int max_sq[2];                  // largest directed squared distance a->b, b->a
    unsigned int lo_inv[3];                  // per axis: max of (kMaxExtent - coordinate) over surface voxels
    unsigned int hi_p1[3];                   //           max of (coordinate + 1); zero-initialised: empty box
    unsigned int done;                       // blocks of k_directed finished
};

struct Box {
    int lo[3], hi[3];                        // inclusive; lo > hi when both surfaces are empty
};

__device__ __forceinline__ Box read_box(const Counters *c)
{
    Box b;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        b.lo[a] = kMaxExtent - (int)c->lo_inv[a];
        b.hi[a] = (int)c->hi_p1[a] - 1;
    }
    return b;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
    size_t surf, fa, fb, ta, tb, hist, ctr, total;
    long long n_bins;
};

Layout layout(int nx, int ny, int nz)
{
    Layout L;
    const size_t N = (size_t)nx * ny * nz;
    L.n_bins = (long long)(nx - 1) * (nx - 1) + (long long)(ny - 1) * (ny - 1) + (long long)(nz - 1) * (nz - 1) + 1;
    L.surf = 0;
    L.fa = align256(N);
    L.fb = L.fa + align256(4 * N);
    L.ta = L.fb + align256(4 * N);
    L.tb = L.ta + align256(4 * N);
    L.hist = L.tb + align256(4 * N);
    L.ctr = L.hist + align256(8 * (size_t)L.n_bins);
    L.total = L.ctr + align256(sizeof(Counters));
    return L;
}

// One warp per 32-voxel chunk of an image row: lanes along x (coalesced);
// the chunk's row and z-plane are found once per warp.
__global__ void k_surface(int nx, int ny, int nz, const uint8_t *__restrict__ a, const uint8_t *__restrict__ b,
                          int label, uint8_t *__restrict__ surf, Counters *ctr)
{
    const int lane = threadIdx.x & 31;
    const int cpr = (nx + 31) / 32;                           // chunks per row
    const long long chunks = (long long)cpr * ny * nz;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long sy = nx, sz = (long long)nx * ny;
    for (long long wc = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wc < chunks; wc += warps) {
        const int c = (int)(wc % cpr);
        const int row = (int)(wc / cpr);                      // k * ny + j
        const int j = row % ny, k = row / ny;
        const int i = c * 32 + lane;
        const long long v = (long long)row * nx + i;
        unsigned bits = 0;
        if (i < nx) {
            const uint8_t *m[2] = {a, b};
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const uint8_t *M = m[s];
                if (M[v] != label) continue;
                const bool inner = i > 0 && i < nx - 1 && j > 0 && j < ny - 1 && k > 0 && k < nz - 1 &&
                                   M[v - 1] == label && M[v + 1] == label && M[v - sy] == label &&
                                   M[v + sy] == label && M[v - sz] == label && M[v + sz] == label;
                if (!inner) bits |= 1u << s;
            }
            surf[v] = (uint8_t)bits;
        }
        const unsigned ca = __popc(__ballot_sync(FULL, bits & 1u));
        const unsigned cb = __popc(__ballot_sync(FULL, bits & 2u));
        if (ca | cb) {
            const unsigned c3[3] = {(unsigned)i, (unsigned)j, (unsigned)k};
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const unsigned li = __reduce_max_sync(FULL, bits ? (unsigned)kMaxExtent - c3[ax] : 0u);
                const unsigned hp = __reduce_max_sync(FULL, bits ? c3[ax] + 1u : 0u);
                if (lane == 0) {
                    atomicMax(&ctr->lo_inv[ax], li);
                    atomicMax(&ctr->hi_p1[ax], hp);
                }
            }
            if (lane == 0) {
                if (ca) atomicAdd(&ctr->n[0], (unsigned long long)ca);
                if (cb) atomicAdd(&ctr->n[1], (unsigned long long)cb);
            }
        }
    }
}

// One warp per row (j, k) of the box: f[x] = (x - nearest surface position of
// the row)^2, kInf if the row has none; both surfaces; the 32-wide chunks
// that meet the box along x.
__global__ void k_edt_x(int nx, int ny, int nz, const uint8_t *__restrict__ surf, const Counters *__restrict__ ctr,
                        int *__restrict__ fa, int *__restrict__ fb)
{
    const Box bx = read_box(ctr);
    if (bx.lo[0] > bx.hi[0]) return;
    const int by = bx.hi[1] - bx.lo[1] + 1;
    const int c_first = (bx.lo[0] / 32) * 32, c_last = (bx.hi[0] / 32) * 32;
    const int lane = threadIdx.x & 31;
    const unsigned upto = lane == 31 ? FULL : ((2u << lane) - 1u);   // positions <= lane
    const unsigned from = ~((1u << lane) - 1u);                      // positions >= lane
    const long long rows = (long long)by * (bx.hi[2] - bx.lo[2] + 1);
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
        const int j = bx.lo[1] + (int)(r % by), k = bx.lo[2] + (int)(r / by);
        const long long base = ((long long)k * ny + j) * nx;
        int last[2] = {-kInf, -kInf};
        for (int c = c_first; c <= c_last; c += 32) {   // nearest surface position at or left of x
            const int x = c + lane;
            const unsigned s = x < nx ? surf[base + x] : 0u;
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const unsigned bm = __ballot_sync(FULL, (s >> m) & 1u);
                const unsigned left = bm & upto;
                const int pos = left ? c + 31 - __clz(left) : last[m];
                if (x < nx) (m == 0 ? fa : fb)[base + x] = x - pos;
                if (bm) last[m] = c + 31 - __clz(bm);
            }
        }
        int next[2] = {2 * kInf, 2 * kInf};
        for (int c = c_last; c >= c_first; c -= 32) {   // and at or right of x
            const int x = c + lane;
            const unsigned s = x < nx ? surf[base + x] : 0u;
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const unsigned bm = __ballot_sync(FULL, (s >> m) & 1u);
                const unsigned right = bm & from;
                const int pos = right ? c + __ffs(right) - 1 : next[m];
                if (x < nx) {
                    int *f = m == 0 ? fa : fb;
                    const int d = min(f[base + x], pos - x);
                    f[base + x] = d < kInf ? d * d : kInf;
                }
                if (bm) next[m] = c + __ffs(bm) - 1;
            }
        }
    }
}

// f_out at (i, line position j, o) = min over q of f_in(i, q, o) + (j - q)^2
// inside the box: line axis la (element stride ls), other axis oa (block
// row o, stride os), i along x (stride 1).  Block: 32 x-neighbours x
// kLineThreadsY; blocks outside the box return at once.  blockIdx.z picks
// the surface: both transforms advance in one launch.
__global__ void k_edt_line(int nx, int la, long long ls, int oa, long long os, const Counters *__restrict__ ctr,
                           const int *__restrict__ fin0, int *__restrict__ fout0, const int *__restrict__ fin1,
                           int *__restrict__ fout1)
{
    const int *__restrict__ fin = blockIdx.z ? fin1 : fin0;
    int *__restrict__ fout = blockIdx.z ? fout1 : fout0;
    extern __shared__ int col[];                       // [line extent of the box][32]
    const Box bx = read_box(ctr);
    const int o = blockIdx.y, i0 = blockIdx.x * 32;
    if (o < bx.lo[oa] || o > bx.hi[oa] || i0 > bx.hi[0] || i0 + 31 < bx.lo[0]) return;   // block-uniform
    const int lo = bx.lo[la], n = bx.hi[la] - lo + 1;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = i0 + tx;
    const long long base = (long long)o * os + i;
    for (int q = ty; q < n; q += kLineThreadsY) col[q * 32 + tx] = i < nx ? fin[base + (lo + q) * ls] : kInf;
    __syncthreads();
    if (i >= nx) return;
    for (int j = ty; j < n; j += kLineThreadsY) {
        int best = kInf;
        int q = 0;
        for (; q + 4 <= n; q += 4) {
            const int d0 = j - q, d1 = d0 - 1, d2 = d0 - 2, d3 = d0 - 3;
            best = min(best, col[q * 32 + tx] + d0 * d0);
            best = min(best, col[(q + 1) * 32 + tx] + d1 * d1);
            best = min(best, col[(q + 2) * 32 + tx] + d2 * d2);
            best = min(best, col[(q + 3) * 32 + tx] + d3 * d3);
        }
        for (; q < n; ++q) {
            const int d = j - q;
            best = min(best, col[q * 32 + tx] + d * d);
        }
        fout[base + (lo + j) * ls] = min(best, kInf);
    }
}

// Nearest-rank 95th percentile of each direction from its histogram (a
// chunked block scan), and the outputs.  Run by one whole block; the
// histograms and counters are read from L2, where the atomics landed.
__device__ void select_and_write(long long n_bins, const unsigned *hist, const Counters *ctr, double *out)
{
    __shared__ unsigned long long warp_tot[32];
    __shared__ long long found;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5, nt = blockDim.x, nw = nt >> 5;
    const unsigned long long na = __ldcg(&ctr->n[0]), nb = __ldcg(&ctr->n[1]);
    long long p95[2] = {0, 0};
    for (int dir = 0; dir < 2; ++dir) {
        const unsigned long long n = dir == 0 ? na : nb;
        const unsigned long long r = (95ull * n + 99ull) / 100ull;   // nearest rank, 1-based
        const unsigned *h = hist + dir * n_bins;
        unsigned long long run = 0;
        if (t == 0) found = -1;
        __syncthreads();
        for (long long b0 = 0; b0 < n_bins && n > 0; b0 += nt) {
            const long long bin = b0 + t;
            const unsigned long long own = bin < n_bins ? __ldcg(h + bin) : 0ull;
            unsigned long long c = own;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long u = __shfl_up_sync(FULL, c, o);
                if (lane >= o) c += u;
            }
            if (lane == 31) warp_tot[w] = c;
            __syncthreads();
            unsigned long long before = 0, chunk = 0;
            for (int x = 0; x < nw; ++x) {
                const unsigned long long v = warp_tot[x];
                if (x < w) before += v;
                chunk += v;
            }
            const unsigned long long incl = run + before + c;
            const unsigned long long prev = incl - own;
            if (bin < n_bins && prev < r && incl >= r) found = bin;   // exactly one bin crosses r
            __syncthreads();
            run += chunk;
            if (found >= 0) break;
        }
        p95[dir] = found;
        __syncthreads();
    }
    if (t == 0) {
        if (na == 0 || nb == 0) {
            out[0] = NAN;
            out[1] = NAN;
        } else {
            const unsigned m0 = __ldcg(&ctr->max_sq[0]), m1 = __ldcg(&ctr->max_sq[1]);
            out[0] = sqrt((double)max(m0, m1));
            out[1] = sqrt((double)max(p95[0], p95[1]));
        }
        out[2] = (double)na;
        out[3] = (double)nb;
    }
}

// At every surface voxel of a, the squared distance to b's surface (b's
// transform), and vice versa: maximum and histogram per direction.  The
// last block to finish then selects the percentiles and writes the outputs.
__global__ void __launch_bounds__(256) k_directed(long long N, const uint8_t *__restrict__ surf,
                                                  const int *__restrict__ fa, const int *__restrict__ fb,
                                                  long long n_bins, unsigned *__restrict__ hist, Counters *ctr,
                                                  double *out)
{
    __shared__ bool last;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x) {
        const unsigned s = surf[v];
        if (!s) continue;
        if (s & 1u) {                                   // a voxel of S_a: its distance to S_b
            const int d = fb[v];
            if (d < n_bins) {
                atomicMax(&ctr->max_sq[0], (unsigned)d);
                atomicAdd(hist + d, 1u);
            }
        }
        if (s & 2u) {
            const int d = fa[v];
            if (d < n_bins) {
                atomicMax(&ctr->max_sq[1], (unsigned)d);
                atomicAdd(hist + n_bins + d, 1u);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&ctr->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        select_and_write(n_bins, hist, ctr, out);
    }
}

bool extents_ok(int nx, int ny, int nz)
{
    return nx >= 1 && ny >= 1 && nz >= 1 && nx <= kMaxExtent && ny <= kMaxExtent && nz <= kMaxExtent;
}

// L: the image extent along the line axis (the box is at most that long),
// n_o: along the other axis.
cudaError_t launch_line(int nx, int la, int L, long long ls, int oa, int n_o, long long os, const Counters *ctr,
                        const int *fin0, int *fout0, const int *fin1, int *fout1, cudaStream_t st)
{
    const size_t smem = (size_t)L * 32 * sizeof(int);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_edt_line, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const dim3 grid((unsigned)((nx + 31) / 32), (unsigned)n_o, 2);
    k_edt_line<<<grid, dim3(32, kLineThreadsY), smem, st>>>(nx, la, ls, oa, os, ctr, fin0, fout0, fin1, fout1);
    return cudaGetLastError();
}

}  // namespace

extern "C" size_t morea_surface_distance_workspace(int32_t nx, int32_t ny, int32_t nz)
{
    if (!extents_ok(nx, ny, nz)) return 0;
    return layout(nx, ny, nz).total;
}

extern "C" morea_status morea_surface_distance(int32_t nx, int32_t ny, int32_t nz, const uint8_t *a,
                                               const uint8_t *b, int32_t label, void *work, size_t work_bytes,
                                               double *out, void *stream)
{
    if (!extents_ok(nx, ny, nz) || !a || !b || !work || !out || label < 0 || label > 255) return MOREA_EINVAL;
    const Layout Lo = layout(nx, ny, nz);
    if (work_bytes < Lo.total || (reinterpret_cast<uintptr_t>(work) & 255) != 0) return MOREA_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = static_cast<char *>(work);
    uint8_t *surf = reinterpret_cast<uint8_t *>(w + Lo.surf);
    int *fa = reinterpret_cast<int *>(w + Lo.fa);
    int *fb = reinterpret_cast<int *>(w + Lo.fb);
    int *ta = reinterpret_cast<int *>(w + Lo.ta);
    int *tb = reinterpret_cast<int *>(w + Lo.tb);
    unsigned *hist = reinterpret_cast<unsigned *>(w + Lo.hist);
    Counters *ctr = reinterpret_cast<Counters *>(w + Lo.ctr);
    const long long N = (long long)nx * ny * nz;
    const long long plane = (long long)nx * ny;
    cudaError_t e = cudaMemsetAsync(w + Lo.hist, 0, Lo.total - Lo.hist, st);   // histograms + counters
    if (e != cudaSuccess) return MOREA_ECUDA;
    const int blocks = (int)std::min<long long>((N + 255) / 256, 152LL * 8);
    const long long chunks = (long long)((nx + 31) / 32) * ny * nz;
    k_surface<<<(int)std::min<long long>((chunks + 7) / 8, 152LL * 16), 256, 0, st>>>(nx, ny, nz, a, b, label, surf,
                                                                                     ctr);
    const int row_blocks = (int)std::min<long long>(((long long)ny * nz + 7) / 8, 152LL * 16);
    k_edt_x<<<row_blocks, 256, 0, st>>>(nx, ny, nz, surf, ctr, fa, fb);
    if ((e = cudaGetLastError()) != cudaSuccess) return MOREA_ECUDA;
    // along y: lines (i, ., k), element stride nx, one block row per z-plane; both surfaces
    if ((e = launch_line(nx, 1, ny, nx, 2, nz, plane, ctr, fa, ta, fb, tb, st)) != cudaSuccess) return MOREA_ECUDA;
    // along z: lines (i, j, .), element stride nx*ny, one block row per y
    if ((e = launch_line(nx, 2, nz, plane, 1, ny, nx, ctr, ta, fa, tb, fb, st)) != cudaSuccess) return MOREA_ECUDA;
    k_directed<<<blocks, 256, 0, st>>>(N, surf, fa, fb, Lo.n_bins, hist, ctr, out);
    return cudaGetLastError() == cudaSuccess ? MOREA_OK : MOREA_ECUDA;
}
