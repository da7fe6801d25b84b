"""Host logic of the N > 1 benchmark path on CPU: two gloo ranks agree on the
slowest rank's time, the whole-job throughput counts every rank's units, and
the reference arm runs on rank 0 only (the path shards by solution; the
replicas exchange nothing but the timing)."""

import json
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    r = bench.Ranks("gloo", gpu=False)
    r.barrier()
    step_ms = 100.0 + 50.0 * rank                      # rank 1 is the slow one
    m = r.max(step_ms)
    v = bench.throughput(2688, 10, r.world, m)
    r.barrier()
    r.close()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"rank": r.rank, "world": r.world, "max_ms": m, "value": v}, f)


def test_two_gloo_ranks_take_the_max_time_and_sum_the_units(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"r{i}.json")) for i in range(world)]
    for i, d in enumerate(res):
        assert d["rank"] == i and d["world"] == world
        assert d["max_ms"] == 150.0
        assert d["value"] == pytest.approx(2 * 2688 * 10 / 0.150)


def test_single_process_needs_no_process_group(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    r = bench.Ranks("gloo", gpu=False)
    assert (r.rank, r.world, r.dist) == (0, 1, None)
    assert r.max(3.5) == 3.5
    assert bench.throughput(100, 4, 1, 2000.0) == pytest.approx(200.0)
    r.close()


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload, steps, warmup, gpus = "c1", 1, 0, 2

    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
