"""Host logic of the multi-rank bench (replicas, one per GPU) over gloo on CPU, world size 2: the
max-over-ranks time, the whole-job throughput, and the reference arm running on rank 0 only."""

import argparse
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r "took" 1 + r seconds: every rank must see the slowest rank's time
        t = bench.max_over_ranks(1.0 + rank, dist, "cpu")
        rate = bench.whole_job_rate(1000, world, 4, t)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{t} {rate}\n")
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_world_size_2(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        t, rate = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert t == 2.0
        assert rate == 1000 * 2 * 4 / 2.0


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(argparse.Namespace(steps=1, warmup=0, impl="reference"))
    assert capsys.readouterr().out == ""
