#!/usr/bin/env python
"""Benchmark of batched MOREA objective evaluation on GB300.

Workload (one "step" = one GOMEA generation of the 128x128x96 FP32 problem):
  * a full evaluation of the population (128 solutions, 2304 tets, both image
    sides, continuous guidance over 1000 contour pairs), then
  * 20 rounds of partial re-evaluation, one request per solution per round
    (breadth-first mesh neighbourhoods of 4-32 points moved on both meshes),
    each round followed by a commit of a seeded accept mask.
  = 128 + 20 x 128 = 2688 solution evaluations per step.

Prints one JSON line (rank 0).  `value` is solution-evals/s with all inputs
resident on the device; `e2e` is the same metric through the C ABI with
host (pinned) inputs copied in and objectives copied out inside the timed
region.  `roofline` reports the hot kernel (rasterise + sample) against the
measured HBM copy bandwidth on algorithmic bytes (2 x 4 B per voxel visit).
`cpu_baseline` is the FP64 oracle on the host cores over a bounded sample.

`--impl reference` times the oracle (the plain CPU restatement of the
method) on the same workload, as the reference arm.
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
BYTES_PER_VISIT_F32 = 8          # own voxel + one amortised voxel of the other image, 4 B each
L2_FLUSH_BYTES = 512 << 20       # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload(seed_offset=0):
    import synth
    p = synth.make_c1()
    adj = synth.vertex_adjacency(p.tets, p.n_points)
    rounds = synth.partial_requests(p, adj, ROUNDS, 4, 32, 1.0, 3 + seed_offset)
    rng = np.random.default_rng(4 + seed_offset)
    accept = [(rng.random(p.n_solutions) < 0.5).astype(np.uint8) for _ in range(ROUNDS)]
    return p, rounds, accept


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

def oracle_sample(orc, p, rounds, cores):
    """Time the FP64 oracle on a bounded sample of the step: `cores` full
    evaluations and 4 x `cores` partial evaluations of the first round, run
    over `cores` threads (each oracle call releases the GIL).  Returns
    (evals/s for the step's mix of 128 full + 2560 partial evaluations,
    description, seconds per full, seconds per partial)."""
    n_full = max(cores, 2)
    sols = list(range(n_full))
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(cores) as ex:
        base = list(ex.map(lambda i: orc.eval(p.sol_src[i], p.sol_tgt[i]), sols))
    t_full = (time.perf_counter() - t0) / n_full          # wall time per full evaluation at `cores` threads
    reqs = []
    rd = rounds[0]
    off = rd["chg_off"]
    for i in sols:
        ids = rd["chg_pts"][off[i]:off[i + 1]]
        ns, nt = p.sol_src[i].copy(), p.sol_tgt[i].copy()
        ns[ids] = rd["chg_src"][off[i]:off[i + 1]]
        nt[ids] = rd["chg_tgt"][off[i]:off[i + 1]]
        reqs.append((i, ns, nt, ids))
    reqs = reqs * 4
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(cores) as ex:
        list(ex.map(lambda r: orc.eval_partial(p.sol_src[r[0]], p.sol_tgt[r[0]], r[1], r[2], r[3], base[r[0]]),
                    reqs))
    t_part = (time.perf_counter() - t0) / len(reqs)
    n_sol = p.n_solutions
    step_s = n_sol * t_full + ROUNDS * n_sol * t_part
    evals = n_sol + ROUNDS * n_sol
    desc = (f"{n_full} full + {len(reqs)} partial oracle evaluations of the 128x128x96 problem on {cores} threads; "
            f"{t_full * 1e3:.0f} ms/full, {t_part * 1e3:.1f} ms/partial (wall, parallel); step = 128 full + 2560 partial")
    return evals / step_s, desc, t_full, t_part


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    cores = os.cpu_count() or 1
    p, rounds, accept = workload()
    orc = oracle.Oracle(p)
    per_step = []
    desc = ""
    for s in range(args.warmup + args.steps):
        v, desc, tf, tp = oracle_sample(orc, p, rounds, cores)
        if s >= args.warmup:
            per_step.append(v)
    value = float(np.mean(per_step))
    evals = p.n_solutions * (1 + ROUNDS)
    line = {
        "metric": "solution-evals/sec (full & partial)", "value": value, "unit": "solution-evals/s",
        "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": evals / value * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "c1: 128x128x96 f32, 567 pts / 2304 tets, population 128, 20 partial rounds",
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "solution-evals/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "solution-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2303_04873_gb300 import build as _b
    _b.build()
    from paper_2303_04873_gb300 import morea

    # the oracle sample runs first, on host threads, before any GPU work
    p, rounds, accept = workload()
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        cores = os.cpu_count() or 1
        v, desc, tf, tp = oracle_sample(oracle.Oracle(p), p, rounds, cores)
        cpu = {"value": v, "unit": "solution-evals/s", "cores": cores, "kind": "oracle", "sample": desc}

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

    launches_per_step = 4 + ROUNDS * 4
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
    total_ms = float(sum(step_ms))
    if dist is not None:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    evals_per_step = n * (1 + ROUNDS)
    value = world * evals_per_step * args.steps / (total_ms / 1e3)
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

    def e2e_step():
        d_src.copy_(h_src, non_blocking=True)
        d_tgt.copy_(h_tgt, non_blocking=True)
        for q, hq in zip(dR, hR):
            for k in q:
                q[k].copy_(hq[k], non_blocking=True)
        for a, ha in zip(dA, hA):
            a.copy_(ha, non_blocking=True)
        step(d_src, d_tgt, dR, dA)
        for h, d in zip(h_out_full, out_full):
            h.copy_(d, non_blocking=True)
        for ho, do in zip(h_out_part, out_part):
            for h, d in zip(ho, do):
                h.copy_(d, non_blocking=True)

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
    e2e_total = float(sum(e2e_ms))
    if dist is not None:
        t = torch.tensor([e2e_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())
    e2e_value = world * evals_per_step * args.steps / (e2e_total / 1e3)

    peak, peak_kind = peaks()
    achieved = visits_per_step * args.steps * BYTES_PER_VISIT_F32 / (raster_ms / 1e3) / 1e9
    line = {
        "metric": "solution-evals/sec (full & partial)", "value": value, "unit": "solution-evals/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "c1: 128x128x96 f32 images, 567 pts / 2304 tets, population 128, "
                               "1 full eval + 20 partial rounds (4-32 pts) with commits per step",
                   "evals_per_step": evals_per_step, "l2": "flushed before every timed step (512 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "k_raster (rasterise + map + trilinear + h + guidance)",
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "algorithmic_bytes": f"{BYTES_PER_VISIT_F32} B per voxel visit x {visits_per_step} visits/step",
                     "kernel_ms_per_step": raster_ms / args.steps, "launches": raster_launches},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "solution-evals/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": ck,
        "phases_ms": {"full_eval_128": full_ms, "partial_20_rounds": part_ms,
                      "full_evals_per_s": n / (full_ms / 1e3),
                      "partial_evals_per_s": ROUNDS * n / (part_ms / 1e3)},
        "voxel_visits_per_s": visits_per_step * args.steps / (total_ms / 1e3),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    gp.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
