"""The N > 1 path of bench.py on CPU (gloo, world size 2, 127.0.0.1).

The single solve does not shard: N ranks run N replicas and the reported
time is the maximum over ranks.  The batched form shards: every rank solves
its own seeded batch of 64 boxes, with no collective on the data path; only
the timings meet, in one max-reduction.  These tests run both host-side
pieces under a real two-rank process group.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    import q1elasticity as q
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        # slowest rank wins, element by element
        got = bench.reduce_max(dist, [1.0 + rank, 10.0 - rank, 0.5], "cpu")
        assert got == [float(world), 10.0, 0.5], got
        # every rank its own batch: seeds and instances differ between ranks
        specs = q.batch_specs(64, seed=bench.batch_seed(rank))
        sizes = [sp["n"] for sp in specs]
        gathered = [None] * world
        dist.all_gather_object(gathered, (bench.batch_seed(rank), sizes))
        seeds = [g[0] for g in gathered]
        assert len(set(seeds)) == world
        assert gathered[0][1] != gathered[1][1]
        if rank == 0:
            assert bench.batch_seed(0) == 2202  # the 1-GPU batch is rank 0's
            with open(out, "w") as f:
                f.write("ok")
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_path(tmp_path):
    out = str(tmp_path / "rank0")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    assert open(out).read() == "ok"


def test_single_rank_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(None, [3, 1.5], "cpu") == [3.0, 1.5]
