"""kl_batch_shard: the grids of a batch distributed across ranks by interior
points (longest-processing-time bin packing), with no communication.

Pinned by properties that hold for any correct implementation of the rule:
the shards partition the batch, the reported loads add up, the largest load
stays within the mean plus the largest grid and within Graham's
(4/3 - 1/(3m)) bound of the optimum (found by brute force on small cases),
and two gloo ranks that compute their shards independently agree."""

from __future__ import annotations

import itertools
import json
import os
import socket
import sys

import numpy as np
import pytest

from paper_2303_12374_gb300 import kl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _shards(points, world):
    return [kl.kl_batch_shard(points, world, r) for r in range(world)]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_partition_and_mean_bound(seed, world):
    rng = np.random.default_rng(seed)
    points = [int(x) for x in rng.integers(1, 10**6, size=int(rng.integers(1, 70)))]
    sh = _shards(points, world)
    owned = sorted(i for idx, _ in sh for i in idx)
    assert owned == list(range(len(points)))
    for idx, load in sh:
        assert idx == sorted(idx) and load == sum(points[i] for i in idx)
    loads = [load for _, load in sh]
    assert max(loads) <= sum(points) / world + max(points)


def _optimum(points, world):
    best = None
    for assign in itertools.product(range(world), repeat=len(points)):
        loads = [0] * world
        for p, r in zip(points, assign):
            loads[r] += p
        best = max(loads) if best is None else min(best, max(loads))
    return best


@pytest.mark.parametrize("seed", range(12))
def test_graham_bound_against_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    world = int(rng.integers(2, 4))
    points = [int(x) for x in rng.integers(1, 50, size=int(rng.integers(world + 1, 8)))]
    lpt = max(load for _, load in _shards(points, world))
    opt = _optimum(points, world)
    assert opt <= lpt <= (4 / 3 - 1 / (3 * world)) * opt + 1e-9


def test_worst_case_of_the_rule():
    # the classical instance where the rule takes 4/3 - 1/(3m) of the optimum (m = 2)
    points = [3, 3, 2, 2, 2]
    assert max(load for _, load in _shards(points, 2)) == 7 and _optimum(points, 2) == 6


def test_edge_cases_and_errors():
    assert kl.kl_batch_shard([], 3, 1) == ([], 0)
    assert _shards([5, 5], 4) == [([0], 5), ([1], 5), ([], 0), ([], 0)]
    assert kl.kl_batch_shard([4, 4, 4], 1, 0) == ([0, 1, 2], 12)
    for pts, world, rank in (([1], 0, 0), ([1], 2, 2), ([1], 2, -1), ([-1], 1, 0)):
        with pytest.raises(kl.KLError) as e:
            kl.kl_batch_shard(pts, world, rank)
        assert e.value.status == -1


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2303_12374_gb300 import kl as klr, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = synth.WORKLOADS["batch64_uneven"]
    sizes = synth.batch_sizes(synth.seed_of(spec["index"]), spec["count"])
    points = [nx * ny * nz for nx, ny, nz in sizes]
    mine, load = klr.kl_batch_shard(points, world, rank)     # no data exchanged for this
    everyone = [None] * world
    dist.all_gather_object(everyone, (mine, load))            # only to check the result
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump({"points": points, "all": everyone}, fh)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_batch_workload(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert res[0]["all"] == res[1]["all"]
    points = res[0]["points"]
    shards = res[0]["all"]
    assert sorted(i for idx, _ in shards for i in idx) == list(range(len(points)))
    loads = [load for _, load in shards]
    assert sum(loads) == sum(points)
    assert max(loads) - min(loads) <= max(points)
