// The sampled estimator of App. A.2 (estimator SAMPLED): instead of the voxel
// centres inside a tet copy, N = floor(rate * volume + 1/2) points drawn
// uniformly in barycentric coordinates, lambda_d = e_d / sum e with
// e_d = -log u_d and u the copy's digitally shifted 4-D Sobol point.  Both
// images are sampled trilinearly at p (own copy) and T(p) (other copy, same
// lambda), and the continuous guidance term uses the own distance map at p.
//
// One warp per (entry, side) item.  Lane l takes a contiguous block of the
// copy's points, so consecutive Gray-code indices differ in one bit and the
// next Sobol point is one XOR per dimension (Antonov-Saleev).  The shifts
// come from the copy's snapped coordinates (FNV-1a, then splitmix64), so a
// copy gets the same points in full and partial evaluations.  Per-item sums
// are compensated FP32; the sample count is the record's voxel count.
#include "image_ops.cuh"

namespace morea {

namespace {

constexpr long long kMaxSamples = 1LL << 24;

// Direction numbers of the first four Sobol dimensions (written by
// sample_setup): 0 is the van der Corput sequence, 1-3 follow the primitive
// polynomials x + 1, x^2 + x + 1, x^3 + x + 1 with initial numbers {1},
// {1, 3}, {1, 3, 1}.
__constant__ uint32_t c_sobol[4][32];

__device__ __forceinline__ uint32_t sobol_natural(uint32_t n, int d)
{
    uint32_t x = 0;
    for (int b = 0; n != 0; ++b, n >>= 1)
        if (n & 1u) x ^= c_sobol[d][b];
    return x;
}

// Digital shifts of a copy: FNV-1a (64-bit) over its 12 snapped coordinates
// as little-endian int32 words, then the high halves of the first four
// splitmix64 outputs from that state.
__device__ __forceinline__ void copy_shifts(const int4 *q, uint32_t shift[4])
{
    unsigned long long h = 0xcbf29ce484222325ull;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int4 v = q[i];
        const uint32_t w[3] = {(uint32_t)v.x, (uint32_t)v.y, (uint32_t)v.z};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int byte = 0; byte < 4; ++byte) {
                h ^= (w[a] >> (8 * byte)) & 0xffu;
                h *= 0x100000001b3ull;
            }
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        h += 0x9E3779B97F4A7C15ull;
        unsigned long long z = h;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        shift[d] = (uint32_t)(z >> 32);
    }
}

template <typename TI, bool GUIDE>
__global__ void __launch_bounds__(kBlock, 4) k_sample(const DevProblem *__restrict__ probs,
                                                     const WorkEntry *__restrict__ entries,
                                                     const RasterSetup *__restrict__ setup,
                                                     RasterOut *__restrict__ rout, const int *n_entries_dev,
                                                     int n_entries_host, int chunk, int *queue)
{
    using QT = typename QuadOf<TI>::T;
    // per warp: vertex 0 and edge vectors of the own (0..3) and the other
    // copy (4..7), voxel units, read by every sample from shared memory
    __shared__ float4 geo[kBlock / 32][8];
    float4 *G4 = geo[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int n_ent = n_entries_dev ? min(*n_entries_dev, n_entries_host) : n_entries_host;
    run_items(2 * n_ent, chunk, queue + kQueueRaster, [&](const int item) {
        const int side = item >= n_ent ? 1 : 0;      // all source sides first, then all target sides
        const int e = item - side * n_ent;
        const int valid = setup[2 * (size_t)e + side].valid;
        float s_img = 0.0f, c_img = 0.0f, s_g = 0.0f, c_g = 0.0f;
        long long n = 0;
        if (valid & 1) {
            const WorkEntry &we = entries[e];
            const DevProblem &P = probs[we.prob];
            const int4 *own = we.q[side], *oth = we.q[1 - side];
            const double D = orient_d(own[0], own[1], own[2], own[3]);
            const double Sd = (double)P.S;
            const double vol = D / (6.0 * Sd * Sd * Sd);
            n = (long long)floor((double)P.rate * vol + 0.5);
            n = min(n, kMaxSamples);
            uint32_t shift[4];
            copy_shifts(own, shift);
            // vertex 0 and edges of both copies in voxel units (exact in FP32)
            if (lane < 8) {
                const int4 *c = lane < 4 ? own : oth;
                const int i = lane & 3;
                const float inv_s = 1.0f / (float)P.S;
                const int4 a = c[i], o = c[0];
                G4[lane] = i == 0 ? make_float4(a.x * inv_s - 0.5f, a.y * inv_s - 0.5f, a.z * inv_s - 0.5f, 0.0f)
                                  : make_float4((a.x - o.x) * inv_s, (a.y - o.y) * inv_s, (a.z - o.z) * inv_s, 0.0f);
            }
            __syncwarp();
            const int nx = P.nx, ny = P.ny, nz = P.nz;
            const QT *qown = (const QT *)P.quad[side];
            const QT *qoth = (const QT *)P.quad[1 - side];
            const long long per = (n + 31) / 32;
            const long long j0 = lane * per, j1 = min(n, j0 + per);
            if (j0 < j1) {
                const uint32_t g0 = (uint32_t)(j0 ^ (j0 >> 1));
                uint32_t x[4];
#pragma unroll
                for (int d = 0; d < 4; ++d) x[d] = sobol_natural(g0, d) ^ shift[d];
                for (long long j = j0; j < j1; ++j) {
                    if (j > j0) {                     // gray(j) = gray(j - 1) ^ (1 << ctz(j))
                        const int b = __ffs((int)j) - 1;
#pragma unroll
                        for (int d = 0; d < 4; ++d) x[d] ^= c_sobol[d][b];
                    }
                    float ed[4], sum = 0.0f;
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        const float u = fmaf((float)x[d], 2.3283064365386963e-10f, 1.1641532182693481e-10f);
                        ed[d] = -logf(u);
                        sum += ed[d];
                    }
                    const float inv = 1.0f / sum;
                    const float l1 = ed[1] * inv, l2 = ed[2] * inv, l3 = ed[3] * inv;
                    const float4 v0 = G4[0], e1 = G4[1], e2 = G4[2], e3 = G4[3];
                    const float px = fmaf(l3, e3.x, fmaf(l2, e2.x, fmaf(l1, e1.x, v0.x)));
                    const float py = fmaf(l3, e3.y, fmaf(l2, e2.y, fmaf(l1, e1.y, v0.y)));
                    const float pz = fmaf(l3, e3.z, fmaf(l2, e2.z, fmaf(l1, e1.z, v0.z)));
                    const float4 w0 = G4[4], f1 = G4[5], f2 = G4[6], f3 = G4[7];
                    const float yx = fmaf(l3, f3.x, fmaf(l2, f2.x, fmaf(l1, f1.x, w0.x)));
                    const float yy = fmaf(l3, f3.y, fmaf(l2, f2.y, fmaf(l1, f1.y, w0.y)));
                    const float yz = fmaf(l3, f3.z, fmaf(l2, f2.z, fmaf(l1, f1.z, w0.z)));
                    const float a = trilin_quad(qown, nx, ny, nz, px, py, pz);
                    const float b = trilin_quad(qoth, nx, ny, nz, yx, yy, yz);
                    kadd(s_img, c_img, (a - b) * (a - b));
                    if (GUIDE) {
                        // groups whose map is below r somewhere on p's cell (exact skip of the rest)
                        const int cx = min((int)fminf(fmaxf(px, 0.0f), (float)(nx - 1)), nx - 2);
                        const int cy = min((int)fminf(fmaxf(py, 0.0f), (float)(ny - 1)), ny - 2);
                        const int cz = min((int)fminf(fmaxf(pz, 0.0f), (float)(nz - 1)), nz - 2);
                        unsigned mk = __ldg(P.bandd[side] + ((size_t)cz * ny + cy) * nx + cx);
                        while (mk) {
                            const int g = __ffs(mk) - 1;
                            mk &= mk - 1;
                            const size_t goff = (size_t)g * ((size_t)nx * ny * nz);
                            const float dg = trilin_plain(P.dmap[side] + goff, nx, ny, nz, px, py, pz);
                            if (dg < P.r) {
                                const float dm = trilin_plain(P.dmap[1 - side] + goff, nx, ny, nz, yx, yy, yz);
                                const float df = dg - dm;
                                kadd(s_g, c_g, P.wgt[g] * (P.r - dg) * P.inv_r * df * df);
                            }
                        }
                    }
                }
            }
        }
        const float e_img = warp_comp_sum(s_img, -c_img);
        const float e_g = GUIDE ? warp_comp_sum(s_g, -c_g) : 0.0f;
        if (lane == 0) {
            RasterOut ro;
            ro.e_img = e_img;
            ro.e_guid = e_g;
            ro.n_vox = (int)n;
            ro.n_gp = 0;
            rout[2 * (size_t)e + side] = ro;
            const int pi = entries[e].prob;
            BatchClock *ck = probs[pi].clock;
            if (ck && atomicAdd(&ck->raster_done[pi], 1) + 1 == ck->raster_total[pi]) ck->t_raster[pi] = global_ns();
        }
    });
}

// 2x2x2 cell maximum of the band masks: bit g of out[idx] is set if the
// group's map is below r at any corner of the trilinear cell starting at idx.
__global__ void k_band_dilate(int nx, int ny, int nz, const uint8_t *__restrict__ band, uint8_t *__restrict__ out)
{
    const long long N = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
        unsigned m = 0;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int xx = min(x + dx, nx - 1), yy = min(y + dy, ny - 1), zz = min(z + dz, nz - 1);
                    m |= band[((size_t)zz * ny + yy) * nx + xx];
                }
        out[i] = (uint8_t)m;
    }
}

template <typename TI>
cudaError_t launch_t(const DevProblem *probs, const DevProblem &hp, const WorkEntry *entries, const RasterSetup *setup,
                     RasterOut *rout, const int *n_dev, int n_host, int grid, int chunk, int *queue, cudaStream_t st)
{
    if (hp.g_mode == MOREA_G_CONTINUOUS && hp.G > 0)
        k_sample<TI, true><<<grid, kBlock, 0, st>>>(probs, entries, setup, rout, n_dev, n_host, chunk, queue);
    else
        k_sample<TI, false><<<grid, kBlock, 0, st>>>(probs, entries, setup, rout, n_dev, n_host, chunk, queue);
    return cudaGetLastError();
}

}  // namespace

cudaError_t sample_setup(cudaStream_t st)
{
    // direction numbers from the primitive polynomials and initial numbers above:
    // m_k = m_{k-s} ^ (m_{k-s} << s) ^ sum_{i<s} a_i (m_{k-i} << i), v_k = m_k 2^(32-k)
    uint32_t v[4][32];
    for (int b = 0; b < 32; ++b) v[0][b] = 1u << (31 - b);
    const int degree[3] = {1, 2, 3}, inner[3] = {0, 1, 1};
    const uint32_t init[3][3] = {{1, 0, 0}, {1, 3, 0}, {1, 3, 1}};
    for (int d = 1; d < 4; ++d) {
        const int s = degree[d - 1];
        uint32_t m[33] = {0};
        for (int k = 1; k <= s; ++k) m[k] = init[d - 1][k - 1];
        for (int k = s + 1; k <= 32; ++k) {
            uint32_t t = m[k - s] ^ (m[k - s] << s);
            for (int i = 1; i < s; ++i)
                if ((inner[d - 1] >> (s - 1 - i)) & 1) t ^= m[k - i] << i;
            m[k] = t;
        }
        for (int k = 1; k <= 32; ++k) v[d][k - 1] = m[k] << (32 - k);
    }
    return cudaMemcpyToSymbolAsync(c_sobol, v, sizeof(v), 0, cudaMemcpyHostToDevice, st);
}

cudaError_t launch_band_dilate(const DevProblem &hp, const uint8_t *band, uint8_t *out, cudaStream_t st)
{
    const long long N = (long long)hp.nx * hp.ny * hp.nz;
    k_band_dilate<<<(int)std::min<long long>((N + 255) / 256, 8192), 256, 0, st>>>(hp.nx, hp.ny, hp.nz, band, out);
    return cudaGetLastError();
}

cudaError_t launch_sample(const DevProblem *probs, const DevProblem &hp, const WorkEntry *entries,
                          const RasterSetup *setup, RasterOut *rout, const int *n_entries_dev, int n_entries_host,
                          int grid, int chunk, int *queue, cudaStream_t st)
{
    if (hp.dtype == MOREA_F16)
        return launch_t<__half>(probs, hp, entries, setup, rout, n_entries_dev, n_entries_host, grid, chunk, queue,
                                st);
    return launch_t<float>(probs, hp, entries, setup, rout, n_entries_dev, n_entries_host, grid, chunk, queue, st);
}

}  // namespace morea
