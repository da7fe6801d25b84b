"""Autotuner for the launch shape of the image/guidance passes.

The hot kernels take two knobs (``morea_set_launch`` /
``morea_batch_set_launch``): blocks per SM (grid size as a multiple of the
SM count) and the scheduling chunk (0 = static striding of (tet, side)
items over warps, > 0 = warps take ``chunk`` items at a time from an atomic
work queue, which evens out uneven tet sizes and uneven problems).  The
tuner times each candidate on the caller's own workload with CUDA events,
keeps the fastest, and caches the choice on disk keyed by the workload's
shape and the GPU, so later runs skip the search.  Results of an evaluation
never depend on the launch shape (per-item arithmetic and reduction order
are fixed), only its speed does.
"""

from __future__ import annotations

import json
import os
from typing import Callable, Dict, Iterable, Optional, Sequence, Tuple

import torch

DEFAULT_CANDIDATES: Tuple[Tuple[int, int], ...] = (
    (4, 0), (8, 0), (16, 0), (4, 1), (8, 1), (8, 2), (8, 4), (16, 2),
)


def cache_path() -> str:
    return os.environ.get("MOREA_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_2303_04873_gb300", "tune.json"))


def _load(path: str) -> Dict[str, list]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, table: Dict[str, list]):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def signature(problems: Sequence, n_sol: Sequence[int], kind: str) -> str:
    """Cache key: GPU name, kind of call and the shape of every problem."""
    dev = torch.cuda.get_device_name(torch.cuda.current_device())
    parts = [f"{p.nx}x{p.ny}x{p.nz}:{p.n_tets}:d{p.dtype}:h{p.h_mode}:g{p.g_mode}"
             f":e{getattr(p, 'estimator', 0)}:n{n}" for p, n in zip(problems, n_sol)]
    return f"{dev}|{kind}|" + ";".join(parts)


def time_call(run: Callable[[], None], reps: int = 5, warmup: int = 2) -> float:
    """Median milliseconds of ``run`` on the current stream (CUDA events)."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        run()
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2]


def tune(target, run: Callable[[], None], key: str, candidates: Iterable[Tuple[int, int]] = DEFAULT_CANDIDATES,
         reps: int = 5, path: Optional[str] = None, force: bool = False):
    """Choose and apply the fastest (blocks_per_sm, chunk) for ``run``.

    ``target`` has ``set_launch(blocks_per_sm, chunk)`` (a Problem or a
    Batch); ``run`` performs one representative evaluation on it.  Returns
    (blocks_per_sm, chunk, {candidate: ms}); cached under ``key``.
    """
    path = path or cache_path()
    table = _load(path)
    if not force and key in table:
        bps, chunk = table[key]["best"]
        target.set_launch(bps, chunk)
        return bps, chunk, {}
    timings = {}
    for bps, chunk in candidates:
        target.set_launch(bps, chunk)
        timings[(bps, chunk)] = time_call(run, reps=reps)
    best = min(timings, key=timings.get)
    target.set_launch(*best)
    table[key] = {"best": list(best), "ms": {f"{b},{c}": t for (b, c), t in timings.items()}}
    _store(path, table)
    return best[0], best[1], timings
