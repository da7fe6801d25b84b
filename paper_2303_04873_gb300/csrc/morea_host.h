// Host-side state of libmorea handles (problems and batches), shared by the
// host translation units.  Not part of the public ABI.
#pragma once

#include <algorithm>
#include <vector>

#include "morea_internal.cuh"

// Launch shape of the image / guidance passes (set by morea_set_launch or
// morea_batch_set_launch, normally chosen by the autotuner).
struct MoreaLaunch {
    int blocks_per_sm = 8;   // grid = blocks_per_sm x SM count
    int chunk = 1;           // 0: static striding of items over warps; > 0: warps take
                             // `chunk` items at a time from an atomic queue
};

struct morea_problem {
    int device = 0;
    morea::DevProblem hp{};
    morea::DevProblem *dp = nullptr;
    std::vector<void *> allocs;
    int V = 0, T = 0, G = 0, max_sol = 0, max_req = 0, max_changed = 0, max_star = 0;
    int cap_entries = 0;
    int *v2t_off = nullptr, *v2t_idx = nullptr;
    morea::WorkEntry *entries = nullptr;
    morea::RasterSetup *setup = nullptr;
    morea::RasterOut *rout = nullptr;
    int2 *bandrows = nullptr;
    morea::TetOut *tout = nullptr;
    int *counter = nullptr;
    int *queue = nullptr;                 // work-queue counters + guidance item list (queue_ints)
    morea::ReqInfo *rinfo = nullptr;
    morea_totals *req_delta = nullptr;
    int *req_chg_pts = nullptr;
    int4 *req_chg_q = nullptr;
    int last_nreq = 0;
    double r = 0.0;
    MoreaLaunch launch;
    // instrumentation (morea_profile)
    unsigned prof = 0;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    unsigned long long *visits = nullptr;
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        int cur = 0;
        if (cudaGetDevice(&cur) == cudaSuccess && cur != dev) {
            prev = cur;
            cudaSetDevice(dev);
        }
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <typename Owner, typename T>
cudaError_t dalloc(Owner *p, T **ptr, size_t count)
{
    void *m = nullptr;
    cudaError_t e = cudaMalloc(&m, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return e;
    }
    p->allocs.push_back(m);
    *ptr = (T *)m;
    return cudaSuccess;
}
