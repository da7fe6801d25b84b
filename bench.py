#!/usr/bin/env python
"""Benchmark of batched MOREA objective evaluation on GB300.

Default workload (one "step" = one GOMEA generation of the 256x256x160 FP16
problem, the largest single-GPU configuration):
  * a full evaluation of the population (256 solutions, graded mesh of 1521
    points / 6912 tets, both image sides, continuous guidance), then
  * 20 rounds of partial re-evaluation, one request per solution per round
    (breadth-first mesh neighbourhoods of 4-32 points moved on both meshes),
    each round followed by a commit of a seeded accept mask.
  = 256 + 20 x 256 = 5376 solution evaluations per step.
`--workload c1` runs the same step on the 128x128x96 FP32 problem
(population 128, 2304 tets).

Prints one JSON line (rank 0).  `value` is solution-evals/s with all inputs
resident on the device; `e2e` is the same metric through the C ABI with
host (pinned) inputs copied in and objectives copied out inside the timed
region.  `roofline` reports the hot kernel (rasterise + sample) against the
measured HBM copy bandwidth on algorithmic bytes (2 b per voxel visit, b the
stored bytes per voxel).  `cpu_baseline` is the FP64 oracle on all host
cores and on one thread, each over a mini-step of the same workload.

`--impl reference` times the oracle (the plain CPU restatement of the
method) on mini-steps of the same workload, as the reference arm.
"""

from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

ROUNDS = 20
# algorithmic bytes per voxel visit: the own voxel + one amortised voxel of the
# other image, b bytes each (b = 4 for FP32 storage, 2 for FP16)
L2_FLUSH_BYTES = 512 << 20       # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--generations", type=int, default=200, help="c3: EA generations per run")
    ap.add_argument("--rounds", type=int, default=4, help="c3: mixing rounds per generation")
    ap.add_argument("--epochs", type=int, default=20, help="c3: surrogate training epochs")
    ap.add_argument("--seeds", type=int, default=5, help="c3: EA seeds compared (200, 201, ...)")
    ap.add_argument("--estimator", choices=["voxels", "sampled"], default="voxels",
                    help="c1/c2: voxel centres (default) or the sampled estimator of App. A.2 (1 point per voxel^3)")
    ap.add_argument("--workload", choices=["c1", "c2", "c3", "c3_gomea", "c4", "repair", "surrogate_train", "groups",
                                           "scores", "init", "gomea"],
                    default="c2",
                    help="c2: 256x256x160 f16 graded mesh (the headline); c1: 128x128x96 f32; "
                         "c4: 16 uneven f16 problems in one batched graph launch; "
                         "repair: fold repair of 128 perturbed solutions; "
                         "surrogate_train: training steps of the surrogate network; "
                         "groups: a generation of DSATUR-grouped partial evaluations")
    return ap.parse_args()


WORKLOADS = {
    "c1": ("c1: 128x128x96 f32 images, 567 pts / 2304 tets, population 128, "
           "1 full eval + 20 partial rounds (4-32 pts) with commits per step", 4),
    "c2": ("c2: 256x256x160 f16 images (HU-like), graded 1521 pts / 6912 tets, population 256, "
           "1 full eval + 20 partial rounds (4-32 pts) with commits per step", 2),
}


def workload(seed_offset=0, name="c1", estimator="voxels"):
    import dataclasses
    import synth
    p = synth.make_c1() if name == "c1" else synth.make_c2()
    if estimator == "sampled":
        p = dataclasses.replace(p, estimator=1, sampling_rate=1.0)
    adj = synth.vertex_adjacency(p.tets, p.n_points)
    rounds = synth.partial_requests(p, adj, ROUNDS, 4, 32, 1.0, 3 + seed_offset)
    rng = np.random.default_rng(4 + seed_offset)
    accept = [(rng.random(p.n_solutions) < 0.5).astype(np.uint8) for _ in range(ROUNDS)]
    return p, rounds, accept


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the timed
# image pass (k_raster + k_guidance) per launch, averaged over one step's 21
# launches, from an ncu capture of `bench.py --workload <w> --steps 1` (see
# profiles/).  Valid only while the image kernels and the work-list builder
# are unchanged: the digest covers their source files, and after any change
# the bench reports null until the traffic is re-measured.
TRAFFIC_SOURCES = ("k_raster.cu", "k_tet.cu", "image_ops.cuh", "morea_device.cuh", "morea_internal.cuh")
MEASURED_TRAFFIC = {
    "c2": {"bytes_per_launch": 736972715,
           "sources_sha256": "0ea7f8c9e58c8f80dc21c355dcdd3c51b686e8f22d2d7ba62885e197eb87bade"},
    "c1": {"bytes_per_launch": 126224445,
           "sources_sha256": "0ea7f8c9e58c8f80dc21c355dcdd3c51b686e8f22d2d7ba62885e197eb87bade"},
}


def traffic_digest():
    import hashlib
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2303_04873_gb300", "csrc", name), "rb") as f:
            h.update(hashlib.sha256(f.read()).digest())
    return h.hexdigest()


def measured_traffic(workload):
    rec = MEASURED_TRAFFIC.get(workload)
    if rec is None:
        return None
    return rec["bytes_per_launch"] if traffic_digest() == rec["sources_sha256"] else None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            target = uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-i", target,
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU: the oracle
# ---------------------------------------------------------------------------

def oracle_sample(orc, p, rounds, accept, n_sol, threads):
    """Time the FP64 oracle on a mini-step of the workload: the first
    `n_sol` solutions of the population get the step's own sequence -- a full
    evaluation, then 20 rounds of their partial requests, each round's
    accepted candidates committed as in the GPU step -- run over `threads`
    host threads (each oracle call releases the GIL).  The mix of full and
    partial evaluations (1 : 20) is the step's, so evals/s carries over.
    Returns a dict: evals, seconds (wall), evals/s, ms per full and per
    partial evaluation (wall at this thread count) and a description."""
    sols = list(range(n_sol))
    cur_s = [p.sol_src[i].copy() for i in sols]
    cur_t = [p.sol_tgt[i].copy() for i in sols]
    with cf.ThreadPoolExecutor(threads) as ex:
        t0 = time.perf_counter()
        base = list(ex.map(lambda i: orc.eval(cur_s[i], cur_t[i]), sols))
        t_full = time.perf_counter() - t0
        t1 = time.perf_counter()
        for r in range(ROUNDS):
            rd = rounds[r]
            off = rd["chg_off"]
            reqs = []
            for i in sols:
                ids = rd["chg_pts"][off[i]:off[i + 1]]
                ns, nt = cur_s[i].copy(), cur_t[i].copy()
                ns[ids] = rd["chg_src"][off[i]:off[i + 1]]
                nt[ids] = rd["chg_tgt"][off[i]:off[i + 1]]
                reqs.append((i, ns, nt, ids))
            res = list(ex.map(lambda q: orc.eval_partial(cur_s[q[0]], cur_t[q[0]], q[1], q[2], q[3], base[q[0]]),
                              reqs))
            for (i, ns, nt, _), rr in zip(reqs, res):
                if accept[r][i]:
                    cur_s[i], cur_t[i], base[i] = ns, nt, rr
        t_part = time.perf_counter() - t1
    seconds = t_full + t_part
    evals = n_sol * (1 + ROUNDS)
    desc = (f"mini-step of {n_sol} solutions of the {p.nx}x{p.ny}x{p.nz} problem on {threads} thread(s): "
            f"{n_sol} full + {ROUNDS * n_sol} partial oracle evaluations with commits (the step's 1:{ROUNDS} mix), "
            f"{t_full / n_sol * 1e3:.1f} ms/full, {t_part / (ROUNDS * n_sol) * 1e3:.2f} ms/partial (wall)")
    return {"evals": evals, "seconds": seconds, "value": evals / seconds, "ms_full": t_full / n_sol * 1e3,
            "ms_partial": t_part / (ROUNDS * n_sol) * 1e3, "sample": desc}


def cpu_baselines(orc, p, rounds, accept):
    """The oracle on all host cores (one mini-step of `cores` solutions) and
    on one thread (a mini-step of one solution)."""
    cores = os.cpu_count() or 1
    allc = oracle_sample(orc, p, rounds, accept, min(cores, p.n_solutions), cores)
    one = oracle_sample(orc, p, rounds, accept, 1, 1)
    return {"value": allc["value"], "unit": "solution-evals/s", "cores": cores, "kind": "oracle",
            "sample": allc["sample"],
            "single_thread": {"value": one["value"], "unit": "solution-evals/s", "cores": 1,
                              "sample": one["sample"]}}


def run_reference(args):
    """The reference arm: the oracle as it stands, on all host cores.  The K
    timed steps together run whole mini-steps of the workload (the first
    `cores` solutions through the step's full evaluation and its 20 partial
    rounds with commits, the 1:20 mix of the GPU step): a mini-step's rounds
    are dealt out over consecutive timed steps, the first of them also
    running the full evaluations, with ceil(K / 20) mini-steps in all.  So
    the run's time does not grow with K while its evals/s is that of whole
    mini-steps.  A warm-up step is one partial evaluation of solution 0.
    `ms_per_step` is the measured wall time over K; `extrapolated` projects
    the rate to a step of the whole population."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload not in ("c1", "c2"):
        print(json.dumps({"impl": "reference", "unavailable": f"the oracle arm times the c1/c2 evaluation "
                                                              f"steps, not the {args.workload} workload"}))
        return 0
    import oracle
    cores = os.cpu_count() or 1
    p, rounds, accept = workload(name=args.workload, estimator=args.estimator)
    orc = oracle.Oracle(p)
    n_sol = min(cores, p.n_solutions)
    sols = list(range(n_sol))
    K = max(1, args.steps)
    n_mini = -(-K // ROUNDS)                      # mini-steps covering the K steps
    # step k of mini-step m runs rounds [lo, hi) of it; its first step also the full evaluations
    plan = []
    per = [K // n_mini + (1 if m < K % n_mini else 0) for m in range(n_mini)]
    for m in range(n_mini):
        for k in range(per[m]):
            plan.append((m, k == 0, ROUNDS * k // per[m], ROUNDS * (k + 1) // per[m]))
    base0 = orc.eval(p.sol_src[0], p.sol_tgt[0])
    rd0 = rounds[0]
    ids0 = rd0["chg_pts"][rd0["chg_off"][0]:rd0["chg_off"][1]]
    for _ in range(args.warmup):                  # warm-up: one partial evaluation of solution 0
        ns, nt = p.sol_src[0].copy(), p.sol_tgt[0].copy()
        ns[ids0] = rd0["chg_src"][rd0["chg_off"][0]:rd0["chg_off"][1]]
        nt[ids0] = rd0["chg_tgt"][rd0["chg_off"][0]:rd0["chg_off"][1]]
        orc.eval_partial(p.sol_src[0], p.sol_tgt[0], ns, nt, ids0, base0)
    secs, evals = [], 0
    t_full = t_part = 0.0
    with cf.ThreadPoolExecutor(cores) as ex:
        for m, first, lo, hi in plan:
            t0 = time.perf_counter()
            if first:
                cur_s = [p.sol_src[i].copy() for i in sols]
                cur_t = [p.sol_tgt[i].copy() for i in sols]
                base = list(ex.map(lambda i: orc.eval(cur_s[i], cur_t[i]), sols))
                evals += n_sol
                t_full += time.perf_counter() - t0
            t1 = time.perf_counter()
            for r in range(lo, hi):
                rd = rounds[r]
                off = rd["chg_off"]
                reqs = []
                for i in sols:
                    ids = rd["chg_pts"][off[i]:off[i + 1]]
                    ns, nt = cur_s[i].copy(), cur_t[i].copy()
                    ns[ids] = rd["chg_src"][off[i]:off[i + 1]]
                    nt[ids] = rd["chg_tgt"][off[i]:off[i + 1]]
                    reqs.append((i, ns, nt, ids))
                res = list(ex.map(lambda q: orc.eval_partial(cur_s[q[0]], cur_t[q[0]], q[1], q[2], q[3],
                                                             base[q[0]]), reqs))
                for (i, ns, nt, _), rr in zip(reqs, res):
                    if accept[r][i]:
                        cur_s[i], cur_t[i], base[i] = ns, nt, rr
                evals += n_sol
            t_part += time.perf_counter() - t1
            secs.append(time.perf_counter() - t0)
    total_s = float(sum(secs))
    value = evals / total_s
    full_evals = p.n_solutions * (1 + ROUNDS)
    desc = (f"{n_mini} mini-step(s) of {n_sol} solutions of the {p.nx}x{p.ny}x{p.nz} problem on {cores} "
            f"thread(s), dealt over the {K} timed steps: {n_mini * n_sol} full + {n_mini * ROUNDS * n_sol} "
            f"partial oracle evaluations with commits (the step's 1:{ROUNDS} mix), "
            f"{t_full / (n_mini * n_sol) * 1e3:.1f} ms/full, {t_part / (n_mini * ROUNDS * n_sol) * 1e3:.2f} "
            f"ms/partial (wall)")
    line = {
        "metric": "solution-evals/sec (full & partial)", "value": value, "unit": "solution-evals/s",
        "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_s / K * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][0], "estimator": args.estimator, "l2": "n/a (CPU)",
                   "step": f"1/{per[0]} of a mini-step of {n_sol} of {p.n_solutions} solutions "
                           f"({n_sol * (1 + ROUNDS)} evaluations per mini-step)",
                   "warmup_step": "one partial oracle evaluation of solution 0"},
        "extrapolated": {"ms_per_step": full_evals / value * 1e3, "evals_per_step": full_evals,
                         "note": "the measured rate projected to a step of the whole population"},
        "cpu_baseline": {"value": value, "unit": "solution-evals/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "solution-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------

class Ranks:
    """One process per GPU under torchrun: rank and world size from the
    environment, a process group when world > 1, a barrier that also drains
    the GPU, and the maximum of a time over ranks.  The replicas exchange
    nothing else (the work shards by solution)."""

    def __init__(self, backend: str = "nccl", gpu: bool = True):
        self.gpu = gpu
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.backend = backend
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        import torch
        if self.dist is not None:
            self.dist.barrier()
        if self.gpu:
            torch.cuda.synchronize()

    def max(self, x: float) -> float:
        if self.dist is None:
            return float(x)
        import torch
        dev = torch.device("cuda", self.local) if self.backend == "nccl" else torch.device("cpu")
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


def throughput(units_per_rank_step: float, steps: int, world: int, max_ms: float) -> float:
    """Whole-job units/s: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank_step * steps / (max_ms / 1e3)


def run_ours(args):
    import torch
    ranks = Ranks("nccl")
    rank, world, local = ranks.rank, ranks.world, ranks.local
    torch.cuda.set_device(local)
    barrier = ranks.barrier

    from paper_2303_04873_gb300 import build as _b
    _b.build()
    from paper_2303_04873_gb300 import morea

    # the oracle sample runs first, on host threads, before any GPU work
    p, rounds, accept = workload(name=args.workload, estimator=args.estimator)
    bytes_per_visit = 2 * WORKLOADS[args.workload][1]
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        cpu = cpu_baselines(oracle.Oracle(p), p, rounds, accept)

    n = p.n_solutions
    gp = morea.Problem(p, max_solutions=n, max_requests=n, max_changed=32)
    dev = torch.device("cuda", local)
    src = torch.as_tensor(p.sol_src).to(dev)
    tgt = torch.as_tensor(p.sol_tgt).to(dev)
    R = [{k: torch.as_tensor(v).to(dev) for k, v in rd.items()} for rd in rounds]
    A = [torch.as_tensor(a).to(dev) for a in accept]
    out_full = (torch.empty((n, 3), dtype=torch.float64, device=dev), torch.empty(n, dtype=torch.uint8, device=dev),
                torch.empty(n, dtype=torch.float64, device=dev))
    out_part = [(torch.empty((n, 3), dtype=torch.float64, device=dev), torch.empty(n, dtype=torch.uint8, device=dev),
                 torch.empty(n, dtype=torch.float64, device=dev)) for _ in range(ROUNDS)]
    stream = torch.cuda.current_stream()

    def step(s_src, s_tgt, reqs, acc):
        gp.eval_full(s_src, s_tgt, out=out_full, stream=stream)
        for r in range(ROUNDS):
            q = reqs[r]
            gp.eval_partial(q["slot"], q["chg_off"], q["chg_pts"], q["chg_src"], q["chg_tgt"], out=out_part[r],
                            stream=stream)
            gp.commit_partial(acc[r], stream=stream)

    # launch shape of the hot passes: autotuned on this workload (untimed, cached)
    from paper_2303_04873_gb300 import autotune
    tune_key = autotune.signature([gp], [n], f"step:{args.workload}")
    bps, chunk, _ = autotune.tune(gp, lambda: step(src, tgt, R, A), tune_key, reps=3)
    cont = p.g_mode == 0                      # continuous guidance adds one kernel per evaluation
    launches_per_step = (5 + int(cont)) + ROUNDS * (5 + int(cont))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        step(src, tgt, R, A)
    torch.cuda.synchronize()
    # voxel visits per step (deterministic: every step restarts from the same population)
    gp.profile(2)
    step(src, tgt, R, A)
    torch.cuda.synchronize()
    _, _, visits_per_step = gp.profile_read()
    gp.profile(0)
    # split timing of the two phases (untimed diagnostics)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    flush.zero_()
    ev[0].record(stream)
    gp.eval_full(src, tgt, out=out_full, stream=stream)
    ev[1].record(stream)
    for r in range(ROUNDS):
        q = R[r]
        gp.eval_partial(q["slot"], q["chg_off"], q["chg_pts"], q["chg_src"], q["chg_tgt"], out=out_part[r],
                        stream=stream)
        gp.commit_partial(A[r], stream=stream)
    ev[2].record(stream)
    torch.cuda.synchronize()
    full_ms = ev[0].elapsed_time(ev[1])
    part_ms = ev[1].elapsed_time(ev[2])

    # ---- timed region: device-resident inputs ----
    clocks = ClockSampler(local)
    gp.profile(1)
    step_ms = []
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(src, tgt, R, A)
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
    barrier()
    raster_ms, raster_launches, _ = gp.profile_read()
    gp.profile(0)
    ck = clocks.stop()
    total_ms = ranks.max(float(sum(step_ms)))
    evals_per_step = n * (1 + ROUNDS)
    value = throughput(evals_per_step, args.steps, world, total_ms)
    assert gp.device_status() == 0

    # ---- e2e through the C ABI with host buffers ----
    pin = lambda t: t.cpu().pin_memory()
    h_src, h_tgt = pin(src), pin(tgt)
    hR = [{k: pin(v) for k, v in q.items()} for q in R]
    hA = [pin(a) for a in A]
    h_out_full = [torch.empty_like(t, device="cpu").pin_memory() for t in out_full]
    h_out_part = [[torch.empty_like(t, device="cpu").pin_memory() for t in o] for o in out_part]
    h2d = (h_src.numel() * 4 + h_tgt.numel() * 4 + sum(v.numel() * v.element_size() for q in hR for v in q.values())
           + sum(a.numel() for a in hA))
    d2h = sum(t.numel() * t.element_size() for t in out_full) + sum(
        t.numel() * t.element_size() for o in out_part for t in o)
    d_src, d_tgt = torch.empty_like(src), torch.empty_like(tgt)
    dR = [{k: torch.empty_like(v) for k, v in q.items()} for q in R]
    dA = [torch.empty_like(a) for a in A]

    # Copies run on a side stream, pipelined with the evaluation: the inputs of
    # partial round r land while the full evaluation and the earlier rounds
    # run, and each round's outputs are read back while later rounds run.
    # The step ends when its last copy has landed.
    copy_stream = torch.cuda.Stream(device=dev)

    def e2e_step():
        go = torch.cuda.Event()
        go.record(stream)
        ev_in = []
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(go)
            d_src.copy_(h_src, non_blocking=True)
            d_tgt.copy_(h_tgt, non_blocking=True)
            ev_in.append(torch.cuda.Event())
            ev_in[-1].record(copy_stream)
        stream.wait_event(ev_in[0])
        gp.eval_full(d_src, d_tgt, out=out_full, stream=stream)
        with torch.cuda.stream(copy_stream):      # issued after the full evaluation, so it starts at once
            for q, hq, a_, ha in zip(dR, hR, dA, hA):
                for k in q:
                    q[k].copy_(hq[k], non_blocking=True)
                a_.copy_(ha, non_blocking=True)
                ev_in.append(torch.cuda.Event())
                ev_in[-1].record(copy_stream)
        outs = [(out_full, h_out_full)]
        for r in range(ROUNDS):
            ev_out = torch.cuda.Event()
            ev_out.record(stream)
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(ev_out)
                for h, d in zip(*outs[-1][::-1]):
                    h.copy_(d, non_blocking=True)
            stream.wait_event(ev_in[r + 1])
            q = dR[r]
            gp.eval_partial(q["slot"], q["chg_off"], q["chg_pts"], q["chg_src"], q["chg_tgt"], out=out_part[r],
                            stream=stream)
            gp.commit_partial(dA[r], stream=stream)
            outs.append((out_part[r], h_out_part[r]))
        ev_out = torch.cuda.Event()
        ev_out.record(stream)
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(ev_out)
            for h, d in zip(*outs[-1][::-1]):
                h.copy_(d, non_blocking=True)
        stream.wait_stream(copy_stream)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = []
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step()
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    barrier()
    e2e_total = ranks.max(float(sum(e2e_ms)))
    e2e_value = throughput(evals_per_step, args.steps, world, e2e_total)

    peak, peak_kind = peaks()
    achieved = visits_per_step * args.steps * bytes_per_visit / (raster_ms / 1e3) / 1e9
    line = {
        "metric": "solution-evals/sec (full & partial)", "value": value, "unit": "solution-evals/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][0], "estimator": args.estimator,
                   "evals_per_step": evals_per_step, "l2": "flushed before every timed step (512 MiB write)",
                   "launch": {"blocks_per_sm": bps, "chunk": chunk},
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": measured_traffic(args.workload) if args.estimator == "voxels" else None,
                     "traffic_unit": "bytes per launch (ncu, DRAM read + write)",
                     "kernel": ("image pass: k_raster (rasterise + map + trilinear + h) + k_guidance"
                                if args.estimator == "voxels" else
                                "image pass: k_sample (Sobol points + map + 2 trilinear samples + h + guidance)"),
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "algorithmic_bytes": f"{bytes_per_visit} B per visit (voxel or sample point) x "
                                          f"{visits_per_step} visits/step; the guidance band's distance-map "
                                          f"reads are not counted (a lower bound)",
                     "kernel_ms_per_step": raster_ms / args.steps, "launches": raster_launches},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "solution-evals/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": ck,
        "phases_ms": {"full_eval": full_ms, "partial_20_rounds": part_ms,
                      "full_evals_per_s": n / (full_ms / 1e3),
                      "partial_evals_per_s": ROUNDS * n / (part_ms / 1e3)},
        "voxel_visits_per_s": visits_per_step * args.steps / (total_ms / 1e3),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    gp.close()
    ranks.close()
    return 0


def run_batch(args):
    """16 problems of uneven sizes (64^3 .. 192x192x128 f16, 200-1500 points,
    populations 32-256): full evaluation of every population in one batched
    evaluation (one launch per kernel), captured once as a CUDA graph and
    replayed; the launch shape comes from the autotuner."""
    import torch
    import synth
    from paper_2303_04873_gb300 import build as _b
    _b.build()
    from paper_2303_04873_gb300 import autotune, morea
    torch.cuda.set_device(0)
    probs = synth.make_c4()
    gps = [morea.Problem(p) for p in probs]
    batch = morea.Batch(gps)
    dev = torch.device("cuda", 0)
    srcs = [torch.as_tensor(p.sol_src).to(dev) for p in probs]
    tgts = [torch.as_tensor(p.sol_tgt).to(dev) for p in probs]
    outs = morea.Batch.outputs(srcs)
    n_total = sum(p.n_solutions for p in probs)
    key = autotune.signature(gps, [p.n_solutions for p in probs], "batch_full")
    bps, chunk, timings = autotune.tune(batch, lambda: batch.eval_full(srcs, tgts, outs), key)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.capture(srcs, tgts, outs, stream)
        for _ in range(max(3, args.warmup)):
            batch.replay(stream)
    stream.synchronize()
    visits = sum(int(gp.read_totals(p.n_solutions)["n_vox"].sum()) for gp, p in zip(gps, probs))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    replays = max(args.steps, 100)
    clocks = ClockSampler(0)
    lat = []
    per_rec, per_obj = [], []                 # per problem and replay: device completion times (ms)
    for _ in range(replays):
        with torch.cuda.stream(stream):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            batch.replay(stream)
            b.record(stream)
        b.synchronize()
        lat.append(a.elapsed_time(b))
        rec, obj = batch.latency()            # read after the replay's timed region
        per_rec.append(rec)
        per_obj.append(obj)
    ck = clocks.stop()
    lat = np.asarray(lat)
    per_rec, per_obj = np.asarray(per_rec), np.asarray(per_obj)
    mean_ms = float(lat.mean())
    # e2e: host inputs copied into the captured buffers, replay, outputs copied back
    h_src = [s.cpu().pin_memory() for s in srcs]
    h_tgt = [t.cpu().pin_memory() for t in tgts]
    h_out = [[o.cpu().pin_memory() for o in oo] for oo in outs]
    e2e = []
    for _ in range(max(args.steps, 10)):
        with torch.cuda.stream(stream):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for d, h in zip(srcs + tgts, h_src + h_tgt):
                d.copy_(h, non_blocking=True)
            batch.replay(stream)
            for ho, do in zip(h_out, outs):
                for h, d in zip(ho, do):
                    h.copy_(d, non_blocking=True)
            b.record(stream)
        b.synchronize()
        e2e.append(a.elapsed_time(b))
    h2d = sum(t.numel() * 4 for t in h_src + h_tgt)
    d2h = sum(t.numel() * t.element_size() for oo in h_out for t in oo)
    peak, peak_kind = peaks()
    achieved = visits * 4 / (mean_ms / 1e3) / 1e9
    line = {
        "metric": "solution-evals/sec (full & partial)", "value": n_total / (mean_ms / 1e3),
        "unit": "solution-evals/s", "n_gpus": 1, "steps": replays, "warmup": args.warmup,
        "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "c4: 16 problems 64^3..192x192x128 f16, 200-1512 points, populations 32-256 "
                               f"({n_total} solutions), one batched full evaluation per graph replay",
                   "launch": {"blocks_per_sm": bps, "chunk": chunk, "tuned": {f"{k[0]},{k[1]}": v
                                                                            for k, v in timings.items()}},
                   "l2": "flushed before every replay (512 MiB write)"},
        "latency_ms": {"p50": float(np.percentile(per_obj, 50)), "p99": float(np.percentile(per_obj, 99)),
                       "samples": int(per_obj.size),
                       "records_p50": float(np.percentile(per_rec, 50)),
                       "records_p99": float(np.percentile(per_rec, 99)),
                       "replay_p50": float(np.percentile(lat, 50)), "replay_p99": float(np.percentile(lat, 99)),
                       "per_problem_objectives_mean": [float(v) for v in per_obj.mean(0)],
                       "note": "per problem x replay, ms from the batch's first kernel (device %globaltimer): "
                               "p50/p99 = the problem's objectives written, records_* = its last image-pass or "
                               "guidance item done; replay_* = whole graph replay (CUDA events)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "whole batched evaluation (graph replay)",
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "algorithmic_bytes": f"4 B per voxel visit x {visits} visits/replay"},
        "cpu_baseline": None,
        "e2e": {"value": n_total / (float(np.mean(e2e)) / 1e3), "unit": "solution-evals/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": 6 * replays,
        "clocks": ck,
        "voxel_visits_per_s": visits / (mean_ms / 1e3),
    }
    print(json.dumps(line), flush=True)
    return 0


def local_step(p, frac=0.1):
    """Per-vertex move scale: a fraction of the smallest adjacent lattice spacing."""
    out = np.empty(p.n_points)
    axes = [np.unique(p.ref_points[:, a]) for a in range(3)]
    for v, q in enumerate(p.ref_points):
        w = []
        for a in range(3):
            k = int(np.searchsorted(axes[a], q[a]))
            if k > 0:
                w.append(axes[a][k] - axes[a][k - 1])
            if k + 1 < len(axes[a]):
                w.append(axes[a][k + 1] - axes[a][k])
        out[v] = frac * min(w)
    return out


def run_surrogate_ea(args):
    """Surrogate pre-screen on the 1521-point FP16 problem: a plain run (seed
    100) logs ~200k exact evaluations and the network is trained on them.
    Then, for each of `--seeds` seeds (200, 201, ...), a plain run, a
    surrogate-screened run and a randomly screened run (same exact budget as
    the screened one) with the same hypervolume reference point are compared
    on final hypervolume and exact evaluations."""
    import torch
    import synth
    from paper_2303_04873_gb300 import build as _b
    _b.build()
    from paper_2303_04873_gb300 import ea, morea
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    clocks = ClockSampler(0)
    p = synth.make_c2()
    P, V = p.n_solutions, p.n_points
    gp = morea.Problem(p, max_solutions=P, max_requests=P, max_changed=32)
    step = local_step(p)
    orders = ea.bfs_orders(p.tets, V, 32)
    G, R = args.generations, args.rounds
    log = []
    data_run = ea.run(gp, p, G, R, seed=100, step_scale=step, log=log, orders=orders, hv_every=G)
    feats = torch.cat([f for f, _ in log])
    targ = np.concatenate([o for _, o in log])
    ok = np.all(np.isfinite(targ), axis=1)
    feats, targ = feats[torch.as_tensor(np.nonzero(ok)[0]).cuda()].contiguous(), targ[ok]
    del log
    t_train = time.perf_counter()
    net = morea.Mlp(3 * V, 512, 256, 3, max_batch=1024, seed=0)
    tr = ea.train_surrogate(net, feats, targ, epochs=args.epochs, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t_train
    n_samples = int(feats.shape[0])
    del feats
    torch.cuda.empty_cache()
    runs = []
    for sd in range(200, 200 + args.seeds):
        plain = ea.run(gp, p, G, R, seed=sd, step_scale=step, orders=orders, hv_every=10)
        sur = ea.run(gp, p, G, R, seed=sd, step_scale=step, orders=orders, hv_every=10,
                     surrogate=tr["surrogate"], ref=plain["ref"])
        rnd = ea.run(gp, p, G, R, seed=sd, step_scale=step, orders=orders, hv_every=10, random_screen=True,
                     ref=plain["ref"])
        # the plain run's hypervolume when it had used as many exact evaluations as the screened run
        hx = np.array([h[1] for h in plain["history"]], float)
        hv = np.array([h[2] for h in plain["history"]], float)
        runs.append({"seed": sd, "hv_plain": plain["hv"], "hv_surrogate": sur["hv"], "hv_random_screen": rnd["hv"],
                     "hv_ratio": sur["hv"] / plain["hv"],
                     "hv_plain_at_surrogate_budget": float(np.interp(sur["exact"], hx, hv)),
                     "exact_plain": plain["exact"], "exact_surrogate": sur["exact"],
                     "exact_random_screen": rnd["exact"],
                     "history_plain": plain["history"], "history_surrogate": sur["history"]})
    ratios = np.array([r["hv_ratio"] for r in runs])
    exact_ratio = float(np.mean([r["exact_plain"] / r["exact_surrogate"] for r in runs]))
    line = {
        "metric": "surrogate-screened EA: exact-evaluation ratio at final hypervolume",
        "value": exact_ratio, "unit": "x fewer exact evaluations",
        "n_gpus": 1, "higher_is_better": True, "data": "synthetic", "dtype": "bf16 (network) / f32 (evaluator)",
        "config": {"workload": f"c3: 256x256x160 f16, 1521 points / 6912 tets, population {P}, {G} generations x "
                               f"{R} mixing rounds, screen 4x (top 25% exactly evaluated), "
                               f"{args.seeds} seeds",
                   "network": f"{3 * V} -> 512 -> 256 -> 3, BF16 weights, FP32 accumulation, Adam",
                   "screen_score": "sum over objectives of (net(candidate) - net(parent)) / std, lowest 25% kept",
                   "training_samples": n_samples, "epochs": args.epochs, "train_seconds": t_train},
        "hv_ratio_mean": float(ratios.mean()), "hv_ratio_min": float(ratios.min()),
        "hv_ratio_random_screen_mean": float(np.mean([r["hv_random_screen"] / r["hv_plain"] for r in runs])),
        "hv_ratio_plain_at_surrogate_budget_mean": float(np.mean([r["hv_plain_at_surrogate_budget"] / r["hv_plain"]
                                                                 for r in runs])),
        "surrogate_mae": tr["mae"].tolist(), "surrogate_r2": tr["r2"].tolist(),
        "runs": runs,
        "wall_seconds": time.perf_counter() - t0,
    }
    line["clocks"] = clocks.stop()
    print(json.dumps(line), flush=True)
    return 0


def run_surrogate_gomea(args):
    """The surrogate pre-screen with the MO-RV-GOMEA generation driver
    (gomea.py, Sec. 3) on the 1521-point FP16 problem, population 64: a plain
    run (seed 100) logs up to 256 exact evaluations per parallel group and
    generation, the network is trained on them; then, for each of `--seeds`
    seeds (200, ...), a plain run, a screened run (the best-predicted 25 % of
    each group's requests evaluated exactly) and a randomly screened run (the
    same exact budget) from the same initial population and hypervolume
    reference point are compared on final hypervolume and exact evaluations."""
    import torch
    import synth
    from paper_2303_04873_gb300 import build as _b
    _b.build()
    from paper_2303_04873_gb300 import ea, gomea, morea
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    clocks = ClockSampler(0)
    n = 64
    G = args.generations
    p = synth.make_c2(n_sol=1)
    cfg = gomea.GomeaConfig()
    gp = morea.Problem(p, max_solutions=n, max_requests=gomea.max_requests(p, n),
                       max_changed=gomea.max_changed(cfg))
    log = []
    data = gomea.Gomea(gp, p, n, cfg, seed=100, log=log, log_per_group=256)
    for _ in range(G):
        data.step()
    feats = torch.cat([f for f, _ in log])
    targ = np.concatenate([o for _, o in log])
    del log
    t_train = time.perf_counter()
    net = morea.Mlp(3 * p.n_points, 512, 256, 3, max_batch=1024, seed=0)
    tr = ea.train_surrogate(net, feats, targ, epochs=args.epochs, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t_train
    n_samples = int(feats.shape[0])
    del feats
    torch.cuda.empty_cache()
    runs = []
    for sd in range(200, 200 + args.seeds):
        start = gomea.Gomea(gp, p, n, cfg, seed=sd)       # the seed's initial population, shared by its runs
        s0, t0_ = start.S.cpu().numpy(), start.T.cpu().numpy()
        ref = 1.1 * start.obj[~start.folded].max(axis=0)
        res = {}
        for kind in ("plain", "surrogate", "random"):
            run = gomea.Gomea(gp, p, n, cfg, seed=sd, start_src=s0, start_tgt=t0_,
                              surrogate=tr["surrogate"] if kind == "surrogate" else None,
                              random_screen=kind == "random")
            hist = [(0, run.exact, run.hypervolume(ref))]
            for g in range(1, G + 1):
                run.step()
                if g % 10 == 0 or g == G:
                    hist.append((g, run.exact, run.hypervolume(ref)))
            res[kind] = {"hv": hist[-1][2], "exact": run.exact, "history": hist}
        hx = np.array([h[1] for h in res["plain"]["history"]], float)
        hv = np.array([h[2] for h in res["plain"]["history"]], float)
        runs.append({"seed": sd, "hv_plain": res["plain"]["hv"], "hv_surrogate": res["surrogate"]["hv"],
                     "hv_random_screen": res["random"]["hv"],
                     "hv_ratio": res["surrogate"]["hv"] / res["plain"]["hv"],
                     "hv_plain_at_surrogate_budget": float(np.interp(res["surrogate"]["exact"], hx, hv)),
                     "exact_plain": res["plain"]["exact"], "exact_surrogate": res["surrogate"]["exact"],
                     "exact_random_screen": res["random"]["exact"],
                     "history_plain": res["plain"]["history"], "history_surrogate": res["surrogate"]["history"]})
    ratios = np.array([r["hv_ratio"] for r in runs])
    line = {
        "metric": "surrogate-screened MO-RV-GOMEA: exact-evaluation ratio at final hypervolume",
        "value": float(np.mean([r["exact_plain"] / r["exact_surrogate"] for r in runs])),
        "unit": "x fewer exact evaluations", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
        "dtype": "bf16 (network) / f32 (evaluator)",
        "config": {"workload": f"c3 with the generation driver: 256x256x160 f16, 1521 points / 6912 tets, "
                               f"population {n}, 10 clusters, {len(data.groups)} parallel groups of "
                               f"{len(data.el_host)} edge elements, {G} generations, screen 25 % of each group's "
                               f"requests, {args.seeds} seeds",
                   "network": f"{3 * p.n_points} -> 512 -> 256 -> 3, BF16 weights, FP32 accumulation, Adam",
                   "training_samples": n_samples, "epochs": args.epochs, "train_seconds": t_train},
        "hv_ratio_mean": float(ratios.mean()), "hv_ratio_min": float(ratios.min()),
        "hv_ratio_random_screen_mean": float(np.mean([r["hv_random_screen"] / r["hv_plain"] for r in runs])),
        "hv_ratio_plain_at_surrogate_budget_mean": float(np.mean([r["hv_plain_at_surrogate_budget"] / r["hv_plain"]
                                                                 for r in runs])),
        "surrogate_mae": tr["mae"].tolist(), "surrogate_r2": tr["r2"].tolist(),
        "runs": runs, "wall_seconds": time.perf_counter() - t0,
    }
    line["clocks"] = clocks.stop()
    print(json.dumps(line), flush=True)
    gp.close()
    return 0


def run_repair(args):
    """Repair of folded solutions (Sec. 4.3.1) on the 128x128x96 problem: 128
    solutions whose points are perturbed by N(0, 2.5^2) voxels on both meshes,
    so most of them fold; each step restores the folded coordinates (a
    device copy) and repairs them with 64 trials per visited point and at
    most 64 visits per solution.  value = repaired solutions per second."""
    import torch
    import synth
    from paper_2303_04873_gb300 import build as _b
    _b.build()
    from paper_2303_04873_gb300 import morea
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    p = synth.make_c1()
    n, mp = p.n_solutions, 64
    rng = np.random.default_rng(21)
    src0 = torch.as_tensor((p.sol_src + rng.normal(0, 2.5, p.sol_src.shape)).astype(np.float32)).to(dev)
    tgt0 = torch.as_tensor((p.sol_tgt + rng.normal(0, 2.5, p.sol_tgt.shape)).astype(np.float32)).to(dev)
    noise = torch.as_tensor(rng.normal(size=(n, mp, 64, 3)).astype(np.float32)).to(dev)
    gp = morea.Problem(p, max_solutions=n)
    folded0, sev0 = gp.check_folds(src0, tgt0)
    src, tgt = src0.clone(), tgt0.clone()
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        src.copy_(src0)
        tgt.copy_(tgt0)
        moved, sev = gp.repair_folds(src, tgt, noise, mp)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    ms = []
    for _ in range(args.steps):
        src.copy_(src0)
        tgt.copy_(tgt0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        moved, sev = gp.repair_folds(src, tgt, noise, mp)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    ck = clocks.stop()
    total = float(sum(ms))
    folded1, _ = gp.check_folds(src, tgt)
    line = {
        "metric": "repaired solutions/sec", "value": n * args.steps / (total / 1e3), "unit": "solutions/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
        "higher_is_better": True, "data": "synthetic", "dtype": "int64/f64 (exact orientations)",
        "config": {"workload": "repair: 128x128x96, 2304 tets, 128 solutions perturbed N(0, 2.5^2) voxels, "
                               "64 trials per visit, at most 64 visits per solution"},
        "folded_before": int(folded0.sum().item()), "folded_after": int(folded1.sum().item()),
        "severity_before_mean": float(sev0.mean().item()), "severity_after_mean": float(sev.mean().item()),
        "moved_points_per_step": int(moved.sum().item()),
        "gpu_launches": args.steps, "clocks": ck,
    }
    print(json.dumps(line), flush=True)
    gp.close()
    return 0


def run_groups(args):
    """One generation of the paper's parallel partial evaluation (Sec. 4.2.1)
    on the 128x128x96 problem: the edge FOS from the greedy set cover is
    coloured into parallel groups by DSATUR, and each group is one batched
    partial evaluation with a request per (solution, element) (two points
    moved by N(0, 1) on both meshes) followed by a commit of a seeded accept
    mask.  value = partial evaluations per second."""
    import torch
    import synth
    from paper_2303_04873_gb300 import build as _b
    _b.build()
    from paper_2303_04873_gb300 import morea
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    p = synth.make_c1()
    n = p.n_solutions
    el, grp = morea.parallel_groups(p.n_points, p.tets)
    n_groups = int(grp.max()) + 1
    biggest = int(np.bincount(grp).max())
    gp = morea.Problem(p, max_solutions=n, max_requests=n * biggest, max_changed=2)
    gp.eval_full(torch.as_tensor(p.sol_src).to(dev), torch.as_tensor(p.sol_tgt).to(dev))
    rng = np.random.default_rng(3)
    rounds = []
    for g in range(n_groups):
        members = el[grp == g]
        m = len(members)
        slots = np.repeat(np.arange(n, dtype=np.int32), m)
        pts = np.tile(members, (n, 1)).reshape(-1).astype(np.int32)
        off = np.arange(0, 2 * n * m + 1, 2, dtype=np.int32)
        step = rng.normal(0, 1.0, size=(len(pts), 2, 3))
        step[np.repeat(p.fixed_axes[pts][:, None, :], 2, axis=1)] = 0.0
        owner = slots.repeat(2)
        new_s = (p.sol_src[owner, pts] + step[:, 0]).astype(np.float32)
        new_t = (p.sol_tgt[owner, pts] + step[:, 1]).astype(np.float32)
        acc = (rng.random(n * m) < 0.5).astype(np.uint8)
        rounds.append(([torch.as_tensor(a).to(dev) for a in (slots, off, pts, new_s, new_t)],
                       torch.as_tensor(acc).to(dev)))
    n_req = sum(int(r[0][0].shape[0]) for r in rounds)
    outs = [(torch.empty((int(r[0][0].shape[0]), 3), dtype=torch.float64, device=dev),
             torch.empty((int(r[0][0].shape[0]),), dtype=torch.uint8, device=dev),
             torch.empty((int(r[0][0].shape[0]),), dtype=torch.float64, device=dev)) for r in rounds]

    def step_fn():
        for (dv, acc), out in zip(rounds, outs):
            gp.eval_partial(*dv, out=out)
            gp.commit_partial(acc)

    for _ in range(max(3, args.warmup)):
        step_fn()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(0)
    ms = []
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step_fn()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    ck = clocks.stop()
    total = float(sum(ms))
    assert gp.device_status() == 0
    line = {
        "metric": "partial evaluations/sec (parallel groups)", "value": n_req * args.steps / (total / 1e3),
        "unit": "partial-evals/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps, "higher_is_better": True, "data": "synthetic", "dtype": "f32",
        "config": {"workload": f"groups: 128x128x96 f32, 2304 tets, population {n}; {len(el)} edge elements "
                               f"(greedy set cover) in {n_groups} DSATUR groups; one batched partial "
                               f"evaluation + commit per group; {n_req} requests per generation"},
        # per group: partial entries, entry work, image pass, guidance pass, finalize, commit
        "gpu_launches": 6 * n_groups * args.steps, "clocks": ck,
    }
    print(json.dumps(line), flush=True)
    gp.close()
    return 0


def run_gomea(args):
    """MO-RV-GOMEA generations (Sec. 3, 4.2-4.3) on the 128x128x96 problem:
    population 128 from the initialisation noise, 10 clusters, the edge FOS
    in its DSATUR parallel groups; each generation clusters the population
    (host), and per group samples one request per (solution, element) from
    its cluster's distribution (device), evaluates them in one batched
    partial evaluation (device), accepts (host) and commits (device), then
    repairs the folded candidates and evaluates the repaired ones.
    Wall-clock time with the device synchronised around each generation.
    value = partial evaluations per second."""
    import time
    import torch
    import synth
    from paper_2303_04873_gb300 import build as _b
    _b.build()
    from paper_2303_04873_gb300 import morea, gomea
    torch.cuda.set_device(0)
    p = synth.make_c1(n_sol=1)
    n = 128
    cfg = gomea.GomeaConfig()
    gp = morea.Problem(p, max_solutions=n, max_requests=gomea.max_requests(p, n), max_changed=gomea.max_changed(cfg))
    run = gomea.Gomea(gp, p, n, cfg, seed=1)
    ref = 1.1 * run.obj.max(axis=0)
    hv0 = run.hypervolume(ref)
    for _ in range(max(3, args.warmup)):
        run.step()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    ms, reqs, accs = [], 0, 0
    calls0 = run.repair_calls
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = run.step()
        torch.cuda.synchronize()
        ms.append((time.perf_counter() - t0) * 1e3)
        reqs += st["requests"]
        accs += st["accepted"]
    ck = clocks.stop()
    total = float(sum(ms))
    assert gp.device_status() == 0
    line = {
        "metric": "partial evaluations/sec (MO-RV-GOMEA generations)", "value": reqs / (total / 1e3),
        "unit": "partial-evals/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps, "higher_is_better": True, "data": "synthetic", "dtype": "f32/f64",
        "config": {"workload": f"gomea: 128x128x96 f32, 2304 tets, population {n}, 10 clusters, "
                               f"{len(run.groups)} parallel groups of {len(run.el_host)} edge elements; "
                               f"one step = one generation (wall clock, host work included)"},
        "requests_per_generation": reqs / args.steps, "accepted_per_generation": accs / args.steps,
        "repaired_candidates": run.repaired, "repaired_accepted": run.repaired_accepted,
        "hv_start": hv0, "hv_end": run.hypervolume(ref), "archive": int(len(run.archive.pts)),
        # per group: sampling (2 kernels), partial evaluation (entries, entry work, image pass, guidance,
        # finalize), commit, slot objectives; per repair: repair, fold check, partial evaluation (5),
        # commit, slot objectives
        "gpu_launches": 9 * len(run.groups) * args.steps + 9 * (run.repair_calls - calls0), "clocks": ck,
    }
    print(json.dumps(line), flush=True)
    gp.close()
    return 0


def run_init(args):
    """Initialisation noise (Sec. 4.2.2, App. A.5) for the 128x128x96
    problem's population: 128 solutions start from the reference mesh and
    8 Gaussian kernels per mesh (centres uniform in the image, sigma 8-24
    voxels, strength 0.02-0.15) attract the points for up to 50 rounds while
    the mesh stays unfolded.  value = initialised solutions per second."""
    import torch
    import synth
    from paper_2303_04873_gb300 import build as _b
    _b.build()
    from paper_2303_04873_gb300 import morea
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    p = synth.make_c1()
    n, K, R = p.n_solutions, 8, 50
    rng = np.random.default_rng(11)
    box = np.array([p.nx, p.ny, p.nz], np.float64) - 1
    ker = np.concatenate([rng.uniform(0, 1, (n, 2, K, 3)) * box, rng.uniform(8, 24, (n, 2, K, 1)),
                          rng.uniform(0.02, 0.15, (n, 2, K, 1))], -1).astype(np.float32)
    f = p.fixed_axes.astype(np.uint8)
    fixed = torch.as_tensor((f[:, 0] | (f[:, 1] << 1) | (f[:, 2] << 2)).astype(np.uint8)).to(dev)
    ref = torch.as_tensor(np.broadcast_to(p.ref_points.astype(np.float32), (n, p.n_points, 3)).copy()).to(dev)
    kd = torch.as_tensor(ker).to(dev)
    gp = morea.Problem(p, max_solutions=1)
    S, T = ref.clone(), ref.clone()
    for _ in range(max(3, args.warmup)):
        S.copy_(ref)
        T.copy_(ref)
        rounds = gp.init_noise(S, T, kd, R, fixed=fixed)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(0)
    ms = []
    for _ in range(args.steps):
        S.copy_(ref)
        T.copy_(ref)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rounds = gp.init_noise(S, T, kd, R, fixed=fixed)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    ck = clocks.stop()
    total = float(sum(ms))
    folded, _ = gp.check_folds(S, T)
    r = rounds.float()
    line = {
        "metric": "initialised solutions/sec (Gaussian attraction noise)", "value": n * args.steps / (total / 1e3),
        "unit": "solutions/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps, "higher_is_better": True, "data": "synthetic",
        "dtype": "f64 (explicitly rounded) / int64 (exact orientations)",
        "config": {"workload": f"init: 128x128x96, 567 points, 2304 tets, {n} solutions x 2 meshes, {K} kernels "
                               f"per mesh, up to {R} rounds"},
        "rounds_mean": float(r.mean().item()), "rounds_min": int(rounds.min().item()),
        "displacement_mean_voxels": float((torch.cat([S, T]) - ref.repeat(2, 1, 1)).norm(dim=-1).mean().item()),
        "folded_after": int(folded.sum().item()),
        "gpu_launches": args.steps, "clocks": ck,
    }
    print(json.dumps(line), flush=True)
    gp.close()
    return 0


def run_scores(args):
    """Registration scores of a population (the evaluation of Sec. 5) on the
    128x128x96 problem with its five organ masks: per solution, the warped
    label image of both sides and the Hausdorff distance and its 95th
    percentile of every organ on each side (2 warps + 10 surface distances).
    value = scored solutions per second."""
    import torch
    import synth
    from paper_2303_04873_gb300 import build as _b
    _b.build()
    from paper_2303_04873_gb300 import morea
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    p = synth.make_c1(n_sol=32)
    n = p.n_solutions
    la, lb = synth.label_pair((p.nx, p.ny, p.nz), synth.phantom.C1_ELLIPSOIDS, 6.0)
    lab = [torch.as_tensor(la).to(dev), torch.as_tensor(lb).to(dev)]
    n_org = len(synth.phantom.C1_ELLIPSOIDS)
    gp = morea.Problem(p, max_solutions=1)
    S = torch.as_tensor(p.sol_src).to(dev)
    T = torch.as_tensor(p.sol_tgt).to(dev)
    work = torch.empty(morea.surface_distance_workspace(p.nx, p.ny, p.nz), dtype=torch.uint8, device=dev)
    scores = torch.empty((n, 2, n_org, 4), dtype=torch.float64, device=dev)

    def step_fn():
        for i in range(n):
            for side in (0, 1):
                w = gp.warp_labels(S[i], T[i], side, lab[1 - side])
                for o in range(n_org):
                    morea.surface_distance(lab[side], w, o + 1, work=work, out=scores[i, side, o])

    for _ in range(max(3, args.warmup)):
        step_fn()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(0)
    ms = []
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step_fn()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    ck = clocks.stop()
    total = float(sum(ms))
    hd = scores[..., 0].cpu().numpy()
    line = {
        "metric": "scored solutions/sec (warped organ masks, HD and HD95)", "value": n * args.steps / (total / 1e3),
        "unit": "solutions/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps, "higher_is_better": True, "data": "synthetic", "dtype": "int32 (exact)",
        "config": {"workload": f"scores: 128x128x96, 2304 tets, {n} solutions, {n_org} organ masks; per solution "
                               f"2 warped label images + {2 * n_org} surface distances"},
        "hd_mean_voxels": float(np.nanmean(hd)),
        # per solution and side: the warp kernel, then per organ 5 kernels (surface, x pass, y and z
        # passes of both surfaces, directed distances with the selection in the last block)
        "gpu_launches": n * 2 * (1 + n_org * 5) * args.steps, "clocks": ck,
    }
    print(json.dumps(line), flush=True)
    gp.close()
    return 0


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), "measured burst cuBLAS bf16"
    except Exception:
        return 1900.0, "fallback"


def run_surrogate_train(args):
    """Training of the surrogate network 4563 -> 512 -> 256 -> 3 on batches of
    1024 random inputs (Adam, BF16 products on tcgen05, FP32 accumulation);
    value = training samples per second.  The roofline reports the five
    tensor-core products of a step against the measured BF16 peak."""
    import torch
    from paper_2303_04873_gb300 import build as _b
    _b.build()
    from paper_2303_04873_gb300 import morea
    torch.cuda.set_device(0)
    n_in, h1, h2, n_out, B = 4563, 512, 256, 3, 1024
    net = morea.Mlp(n_in, h1, h2, n_out, max_batch=B, seed=0)
    gen = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(B, n_in, device="cuda", generator=gen)
    t = torch.randn(B, n_out, device="cuda", generator=gen)
    kin = net.kin
    flops = 2 * B * (kin * h1 + h1 * h2) + 2 * B * (h2 * h1 + h1 * h2 + h1 * kin)
    for _ in range(max(3, args.warmup)):
        net.train_step(x, t, 1e-4)
    torch.cuda.synchronize()
    reps = max(args.steps, 50)
    clocks = ClockSampler(0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        net.train_step(x, t, 1e-4)
    b.record()
    b.synchronize()
    ck = clocks.stop()
    ms = a.elapsed_time(b) / reps
    peak, kind = bf16_peak()
    achieved = flops / (ms * 1e-3) / 1e12
    line = {
        "metric": "surrogate training samples/sec", "value": B / (ms * 1e-3), "unit": "samples/s",
        "n_gpus": 1, "steps": reps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "data": "synthetic", "dtype": "bf16 (products) / f32 (accumulation, Adam)",
        "config": {"workload": "surrogate training: 4563 -> 512 -> 256 -> 3, batch 1024, Adam"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "peak_kind": kind,
                     "kernel": "the five k_gemm_tc products of a step, timed with the whole step"},
        "status": net.device_status(), "clocks": ck,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.workload == "groups" and args.impl != "reference":
        return run_groups(args)
    if args.workload == "surrogate_train" and args.impl != "reference":
        return run_surrogate_train(args)
    if args.workload == "repair" and args.impl != "reference":
        return run_repair(args)
    if args.workload == "scores" and args.impl != "reference":
        return run_scores(args)
    if args.workload == "init" and args.impl != "reference":
        return run_init(args)
    if args.workload == "gomea" and args.impl != "reference":
        return run_gomea(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c4":
        return run_batch(args)
    if args.workload == "c3":
        return run_surrogate_ea(args)
    if args.workload == "c3_gomea":
        return run_surrogate_gomea(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
