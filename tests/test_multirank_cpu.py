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


# ---- ensemble partition over ranks (the data path of an N-GPU ensemble run)

def _ensemble_members():
    from paper_2512_12934_gb300 import workloads as W

    return [W.tjunction(Wc=wc, length_factor=6, Wd=max(4, wc // 2), side_len=wc, x_side=2 * wc, G12=1.2,
                        Gw=(0.1, -0.1), q_ratio=0.5 + 0.1 * j, M=1.0, u_c=0.02)
            for j, wc in enumerate((8, 12, 9, 14, 10, 11, 8))]


def _ensemble_rank(rank, world, port, out_dir):
    import numpy as np
    import torch.distributed as dist

    from oracle import oracle as O
    from paper_2512_12934_gb300 import ensemble

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", world_size=world, rank=rank)
    try:
        ws = _ensemble_members()
        mine = ensemble.share_of([w.fluid_nodes for w in ws], world, rank)
        results = {}
        for i in mine:           # each rank steps only its own instances (the oracle stands in for the GPU)
            o = O.Oracle2D(ws[i].cfg, ws[i].solid, ws[i].rho, ws[i].u)
            o.step(25)
            rho, u, _ = o.macros()
            results[i] = (rho.tolist(), u.tolist())
        gathered = [None] * world
        dist.all_gather_object(gathered, {"rank": rank, "mine": mine, "results": results})
    finally:
        dist.destroy_process_group()
    if rank == 0:
        with open(os.path.join(out_dir, "ensemble.json"), "w") as f:
            json.dump(gathered, f)


def test_ensemble_instances_split_over_two_gloo_ranks_equal_one_rank(tmp_path):
    """Every instance is stepped by exactly one rank, the shares are balanced
    by fluid nodes, and the gathered per-instance fields equal those of a
    single-rank run bit for bit."""
    pytest.importorskip("torch")
    import numpy as np
    import torch.multiprocessing as mp

    from oracle import oracle as O
    from paper_2512_12934_gb300 import ensemble

    world = 2
    mp.spawn(_ensemble_rank, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True)
    gathered = json.load(open(tmp_path / "ensemble.json"))
    ws = _ensemble_members()
    owned = sorted(i for g in gathered for i in g["mine"])
    assert owned == list(range(len(ws)))
    work = [w.fluid_nodes for w in ws]
    loads = [sum(work[i] for i in g["mine"]) for g in gathered]
    assert max(loads) - min(loads) <= max(work)          # LPT balance bound
    for g in gathered:
        for i, (rho, u) in g["results"].items():
            w = ws[int(i)]
            o = O.Oracle2D(w.cfg, w.solid, w.rho, w.u)
            o.step(25)
            r1, u1, _ = o.macros()
            assert np.array_equal(np.array(rho), r1) and np.array_equal(np.array(u), u1)


def test_partition_is_deterministic_complete_and_balanced():
    from paper_2512_12934_gb300 import ensemble

    work = [5, 9, 1, 7, 3, 3, 8, 2]
    for world in (1, 2, 3, 8, 11):
        shares = ensemble.partition(work, world)
        assert len(shares) == world
        assert sorted(i for s in shares for i in s) == list(range(len(work)))
        assert shares == ensemble.partition(work, world)
        loads = [sum(work[i] for i in s) for s in shares]
        assert max(loads) - min(loads) <= max(work)
