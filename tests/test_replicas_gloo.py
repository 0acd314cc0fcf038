"""Replica runs of the benchmark (torchrun, one rank per GPU): the step has
no exchange between beds, so every rank times its own replica and the job is
timed by its slowest rank.  The host logic is checked here with two gloo
ranks on the CPU: the max over ranks, the whole-job value, and the reference
arm that only rank 0 runs."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 1.0 + 0.5 * rank          # rank 1 is the slower replica
        t = bench._max_over_ranks(local_ms, dist, "cpu")
        q.put((rank, t, bench._job_value(1000, world, t)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, value in got:
        assert t == pytest.approx(1.5)
        assert value == pytest.approx(2 * 1000 / 1.5e-3)


def test_without_process_group_the_local_time_stands():
    import bench
    assert bench._max_over_ranks(2.5, None, "cpu") == 2.5
    assert bench._job_value(100, 1, 2.0) == pytest.approx(5e4)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(warmup=3, steps=1, gpus=2)
    assert bench.run_reference(args) == 0   # returns at once, no work, no output


def test_reference_arm_prints_the_workload_config(monkeypatch, capsys):
    """Both arms print the same `config` (the workload alone); the reference
    arm's line, run here on the small Q1 bed, carries the dict that the GPU
    arm builds from the same workload."""
    import argparse
    import json
    import bench
    from paper_2211_01185_gb300 import synth
    monkeypatch.setenv("RANK", "0")
    name = "q1_8x8x32_2k"
    args = argparse.Namespace(warmup=0, steps=1, gpus=1, workload=name)
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    w = synth.make_workload(name)
    assert line["impl"] == "reference" and line["config"] == bench.workload_config(name, w)
    assert line["config"]["nodes"] == (8 + 1) * (8 + 1) * (32 + 1)
    assert line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
