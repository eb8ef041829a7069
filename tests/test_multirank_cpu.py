"""The benchmark's multi-rank logic on CPU: two gloo ranks agree on the
slowest rank's time, and the whole-job rate counts every rank's units over
it.  (On GPU machines the same helpers run over NCCL; the solver itself runs
one independent replica per rank, with no data-path collective.)"""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    w, r, local = bench.dist_env()
    dist.init_process_group("gloo", init_method="env://", world_size=w, rank=r)
    try:
        elapsed_local = 1.5 + rank  # rank 1 is the slow one
        slowest = bench.max_over_ranks(elapsed_local, dist, "cpu")
        rate = bench.job_rate(100.0, w, slowest)
        dist.barrier()
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"env": [w, r, local], "slowest": slowest, "rate": rate}, f)


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    world = 2
    mp.spawn(_rank, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        d = json.load(open(tmp_path / ("rank%d.json" % r)))
        assert d["env"] == [world, r, r]
        assert d["slowest"] == 2.5
        assert d["rate"] == pytest.approx(world * 100.0 / 2.5)


def test_single_rank_helpers_need_no_process_group():
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.job_rate(129024 * 5000, 1, 0.5) == pytest.approx(129024 * 5000 / 0.5)
