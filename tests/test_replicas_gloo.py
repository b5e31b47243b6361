"""Multi-GPU path of the benchmark (independent replicas, no collective in the data path):
the cross-rank reduction of the timed region and the whole-job value, on two gloo ranks
on the CPU."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_ms, value = bench.aggregate_ranks(100.0 + 50.0 * rank, 3, world)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"t_ms": t_ms, "value": value}, f)


def test_two_replicas_take_the_slowest_rank(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["t_ms"] == pytest.approx(150.0)              # max over ranks
        assert r["value"] == pytest.approx(0.150 / (3 * 2))   # all ranks' solves / slowest time


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(80.0, 4, 1) == (80.0, 0.02)
