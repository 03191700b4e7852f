"""The multi-rank bench path on the CPU: two gloo ranks, as torchrun would run
two replicas.  Every rank solves its own systems with no collective on the
data path; the only exchange is the maximum of the timed region, and the
whole-job value counts every rank's systems over that slowest time."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, world, port, out):
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        ms = 10.0 + 5.0 * rank  # the second rank is the slow one
        ms_max = bench.max_over_ranks_of(ms, dist, "cpu")
        out[rank] = (ms_max, bench.whole_job_rate(ms_max, world, 3, 4))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_count_every_rank():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_replica, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank in (0, 1):
        ms_max, value = res[rank]
        assert ms_max == 15.0
        assert value == pytest.approx(2 * 3 * 4 / 0.015)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks_of(7.5) == 7.5
    assert bench.whole_job_rate(250.0, 1, 1, 5) == pytest.approx(20.0)


def test_reference_arm_prints_only_on_rank_zero(capsys, monkeypatch):
    """Under torchrun the reference arm runs on rank 0 alone; the other ranks
    exit without work or output."""
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(workload="cd2d_64_p4", steps=1, warmup=0, gpus=2, impl="reference")
    bench.run_reference(args)
    assert capsys.readouterr().out == ""


def test_reference_arm_line_keeps_the_contract(capsys, monkeypatch):
    """Rank 0 of the reference arm prints one JSON line with the bench keys,
    the oracle as its CPU baseline and an e2e object without copies."""
    import argparse
    import json

    import bench
    monkeypatch.setenv("RANK", "0")
    import time
    args = argparse.Namespace(workload="cd2d_64_p4", steps=2, warmup=0, gpus=1, impl="reference")
    t0 = time.perf_counter()
    bench.run_reference(args)
    wall = time.perf_counter() - t0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # the steps' reported time is time the run really spent, and one thread ran it
    assert d["ms_per_step"] * d["steps"] / 1e3 <= wall
    assert d["cpu_baseline"]["cores"] == 1
