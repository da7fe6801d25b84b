// Host side of batched multi-problem evaluation (morea_batch_*) and of the
// launch-shape knobs the autotuner sets (morea_set_launch,
// morea_batch_set_launch).
#include <algorithm>
#include <new>
#include <vector>

#include "morea_host.h"

using namespace morea;

struct morea_batch {
    int device = 0;
    std::vector<morea_problem *> probs;
    std::vector<void *> allocs;
    DevProblem *dprobs = nullptr;         // device copy of every problem's DevProblem
    DevProblem hp0{};                     // first problem (kernel variant: storage type, modes)
    WorkEntry *entries = nullptr;
    RasterSetup *setup = nullptr;
    RasterOut *rout = nullptr;
    TetOut *tout = nullptr;
    int2 *bandrows = nullptr;
    int *queue = nullptr;
    long long cap_entries = 0;
    MoreaLaunch launch;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    BatchClock *clock = nullptr;          // completion clock of the last evaluation
};

namespace {

morea_status from_cuda(cudaError_t e) { return e == cudaSuccess ? MOREA_OK : MOREA_ECUDA; }

void drop_graph(morea_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Validates the per-problem arguments and fills the table.
morea_status make_table(const morea_batch *b, const int32_t *n_sol, const float *const *src, const float *const *tgt,
                        double *const *obj, uint8_t *const *folded, double *const *severity, BatchTable &tb)
{
    if (!n_sol || !src || !tgt || !obj || !folded) return MOREA_EINVAL;
    tb = BatchTable{};
    tb.n = (int)b->probs.size();
    long long verts = 0, ents = 0;
    int sols = 0;
    for (int i = 0; i < tb.n; ++i) {
        const morea_problem *p = b->probs[i];
        if (n_sol[i] < 1 || n_sol[i] > p->max_sol || !src[i] || !tgt[i] || !obj[i] || !folded[i])
            return MOREA_EINVAL;
        BatchProb &bp = tb.p[i];
        bp.src = src[i];
        bp.tgt = tgt[i];
        bp.obj = obj[i];
        bp.folded = folded[i];
        bp.severity = severity ? severity[i] : nullptr;
        bp.vert_off = verts;
        bp.entry_off = ents;
        bp.sol_off = sols;
        bp.n_sol = n_sol[i];
        verts += (long long)n_sol[i] * p->V;
        ents += (long long)n_sol[i] * p->T;
        sols += n_sol[i];
    }
    if (ents > b->cap_entries) return MOREA_EINVAL;
    tb.total_verts = verts;
    tb.total_entries = ents;
    tb.total_sols = sols;
    return MOREA_OK;
}

cudaError_t enqueue_batch(morea_batch *b, const BatchTable &tb, cudaStream_t st)
{
    cudaError_t e = launch_batch_snap(b->dprobs, tb, st);
    if (e == cudaSuccess) e = launch_batch_entries(b->dprobs, tb, b->entries, st);
    if (e == cudaSuccess)
        e = launch_entry_work(b->dprobs, b->entries, b->setup, b->tout, nullptr, (int)tb.total_entries, nullptr,
                              st);
    if (e == cudaSuccess) {
        const long long items = 2 * tb.total_entries;
        const int grid = (int)std::min<long long>((long long)sm_count() * b->launch.blocks_per_sm, (items + 7) / 8);
        e = launch_raster(b->dprobs, b->hp0, b->entries, b->setup, b->rout, b->bandrows, nullptr,
                          (int)tb.total_entries, std::max(grid, 1), b->launch.chunk, b->queue, false, b->clock,
                          st);
    }
    if (e == cudaSuccess) e = launch_batch_reduce(b->dprobs, tb, b->tout, b->rout, st);
    return e;
}

}  // namespace

extern "C" {

morea_status morea_batch_destroy(morea_batch *b)
{
    if (!b) return MOREA_OK;
    DeviceGuard g(b->device);
    drop_graph(b);
    cudaError_t first = cudaSuccess;
    for (void *m : b->allocs) {
        cudaError_t e = cudaFree(m);
        if (first == cudaSuccess) first = e;
    }
    delete b;
    return from_cuda(first);
}

morea_status morea_batch_create(morea_problem *const *problems, int32_t n_problems, morea_batch **out)
{
    if (!out) return MOREA_EINVAL;
    *out = nullptr;
    if (!problems || n_problems < 1 || n_problems > kMaxBatch) return MOREA_EINVAL;
    const morea_problem *p0 = problems[0];
    if (!p0) return MOREA_EINVAL;
    long long cap = 0;
    for (int i = 0; i < n_problems; ++i) {
        const morea_problem *p = problems[i];
        if (!p || p->device != p0->device || p->hp.dtype != p0->hp.dtype || p->hp.h_mode != p0->hp.h_mode ||
            p->hp.g_mode != p0->hp.g_mode || p->hp.estimator != p0->hp.estimator)
            return MOREA_EINVAL;
        for (int j = 0; j < i; ++j)
            if (problems[j] == p) return MOREA_EINVAL;
        cap += (long long)p->max_sol * p->T;
    }
    if (cap > (1LL << 30)) return MOREA_EINVAL;
    morea_batch *b = new (std::nothrow) morea_batch();
    if (!b) return MOREA_ENOMEM;
    b->device = p0->device;
    DeviceGuard g(b->device);
    b->probs.assign(problems, problems + n_problems);
    b->hp0 = p0->hp;
    b->cap_entries = cap;
    cudaError_t e = dalloc(b, &b->clock, 1);
    std::vector<DevProblem> hps(n_problems);
    for (int i = 0; i < n_problems; ++i) {
        hps[i] = problems[i]->hp;
        hps[i].clock = b->clock;
    }
    if (e == cudaSuccess) e = cudaMemset(b->clock, 0, sizeof(BatchClock));
    if (e == cudaSuccess) e = dalloc(b, &b->dprobs, n_problems);
    if (e == cudaSuccess) e = dalloc(b, &b->entries, (size_t)cap);
    if (e == cudaSuccess) e = dalloc(b, &b->setup, 2 * (size_t)cap);
    if (e == cudaSuccess) e = dalloc(b, &b->rout, 2 * (size_t)cap);
    if (e == cudaSuccess) e = dalloc(b, &b->tout, (size_t)cap);
    if (e == cudaSuccess && p0->hp.g_mode == MOREA_G_CONTINUOUS && p0->hp.estimator == MOREA_EST_VOXELS)
        e = dalloc(b, &b->bandrows, 2 * (size_t)cap * kBandRowsPerItem);
    if (e == cudaSuccess)
        e = dalloc(b, &b->queue,
                   queue_ints(cap, p0->hp.g_mode == MOREA_G_CONTINUOUS && p0->hp.estimator == MOREA_EST_VOXELS));
    if (e == cudaSuccess)
        e = cudaMemcpy(b->dprobs, hps.data(), sizeof(DevProblem) * n_problems, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        morea_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? MOREA_ENOMEM : MOREA_ECUDA;
    }
    *out = b;
    return MOREA_OK;
}

morea_status morea_batch_eval_full(morea_batch *b, const int32_t *n_sol, const float *const *src_pts,
                                   const float *const *tgt_pts, double *const *obj, uint8_t *const *folded,
                                   double *const *severity, void *stream)
{
    if (!b) return MOREA_EINVAL;
    BatchTable tb;
    morea_status s = make_table(b, n_sol, src_pts, tgt_pts, obj, folded, severity, tb);
    if (s != MOREA_OK) return s;
    DeviceGuard g(b->device);
    return from_cuda(enqueue_batch(b, tb, (cudaStream_t)stream));
}

morea_status morea_batch_capture(morea_batch *b, const int32_t *n_sol, const float *const *src_pts,
                                 const float *const *tgt_pts, double *const *obj, uint8_t *const *folded,
                                 double *const *severity, void *stream)
{
    if (!b || !stream) return MOREA_EINVAL;
    BatchTable tb;
    morea_status s = make_table(b, n_sol, src_pts, tgt_pts, obj, folded, severity, tb);
    if (s != MOREA_OK) return s;
    DeviceGuard g(b->device);
    drop_graph(b);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return MOREA_ECUDA;
    cudaError_t e2 = enqueue_batch(b, tb, st);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(st, &graph);
    if (e2 != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return MOREA_ECUDA;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return MOREA_ECUDA;
    }
    b->graph = graph;
    b->exec = exec;
    return MOREA_OK;
}

morea_status morea_batch_replay(morea_batch *b, void *stream)
{
    if (!b || !b->exec) return MOREA_EINVAL;
    DeviceGuard g(b->device);
    return from_cuda(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
}

morea_status morea_batch_latency(morea_batch *b, double *records_ms, double *objectives_ms)
{
    if (!b || (!records_ms && !objectives_ms)) return MOREA_EINVAL;
    DeviceGuard g(b->device);
    BatchClock ck;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&ck, b->clock, sizeof(ck), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return MOREA_ECUDA;
    for (size_t i = 0; i < b->probs.size(); ++i) {
        const bool done = ck.raster_total[i] > 0 && ck.raster_done[i] == ck.raster_total[i] &&
                          ck.guid_done[i] == ck.guid_total[i] && ck.t_reduce[i] != 0;
        const unsigned long long tr = ck.t_raster[i] > ck.t_guid[i] ? ck.t_raster[i] : ck.t_guid[i];
        if (records_ms) records_ms[i] = done ? (double)(long long)(tr - ck.t0) * 1e-6 : -1.0;
        if (objectives_ms) objectives_ms[i] = done ? (double)(long long)(ck.t_reduce[i] - ck.t0) * 1e-6 : -1.0;
    }
    return MOREA_OK;
}

morea_status morea_batch_set_launch(morea_batch *b, int32_t blocks_per_sm, int32_t chunk)
{
    if (!b || blocks_per_sm < 1 || blocks_per_sm > 64 || chunk < 0 || chunk > 1024) return MOREA_EINVAL;
    b->launch.blocks_per_sm = blocks_per_sm;
    b->launch.chunk = chunk;
    return MOREA_OK;
}

morea_status morea_set_launch(morea_problem *p, int32_t blocks_per_sm, int32_t chunk)
{
    if (!p || blocks_per_sm < 1 || blocks_per_sm > 64 || chunk < 0 || chunk > 1024) return MOREA_EINVAL;
    p->launch.blocks_per_sm = blocks_per_sm;
    p->launch.chunk = chunk;
    return MOREA_OK;
}

}  // extern "C"
