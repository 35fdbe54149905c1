"""The N > 1 path of bench.py on CPU: two gloo ranks (one process each) join
through the torchrun environment, the job time is the slowest rank's and the
whole-job value counts every rank's replica; the reference arm runs on rank 0
only."""

from __future__ import annotations

import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    r, local, w = bench.dist_init(world, backend="gloo")
    my_ms = 10.0 + 5.0 * r                      # rank 1 is the slow one
    job_ms = bench.max_over_ranks(my_ms, w, "cpu")
    value = bench.job_value(w, 1000, 10, job_ms)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as fh:
        json.dump({"rank": r, "local": local, "world": w, "job_ms": job_ms, "value": value}, fh)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, d in enumerate(res):
        assert d["rank"] == r and d["local"] == r and d["world"] == world
        assert d["job_ms"] == 15.0
        # 2 replicas x 1000 points x 10 steps in 15 ms
        assert d["value"] == pytest.approx(2 * 1000 * 10 / 15e-3 / 1e9)


def test_single_process_needs_no_group(monkeypatch):
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_init(1) == (0, 0, 1)
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "REF_SECONDS", 0.5)
    monkeypatch.setattr(bench, "WORKLOAD", "walls256_adv5_diff")   # a grid quick to draw
    args = SimpleNamespace(steps=2, warmup=1, gpus=2)
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""
    monkeypatch.setenv("RANK", "0")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    line = json.loads(buf.getvalue())
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["cores"] == bench.host_threads() >= 1
    assert line["config"]["grid"] == "256x256x256"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_cpu_baseline_reports_one_thread_and_all_cores(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "WORKLOAD", "walls256_adv5_diff")
    cb, _ = bench.cpu_baseline(0.3)
    assert cb["kind"] == "oracle" and cb["value"] > 0
    assert cb["single_thread"]["cores"] == 1
    assert cb["cores"] == bench.host_threads()
    assert cb["host_cpus"] == os.cpu_count()
