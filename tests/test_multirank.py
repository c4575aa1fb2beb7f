"""The benchmark's multi-rank host logic on CPU (gloo, world size 2): the timed region is
the maximum over ranks and the units are summed; the replicas draw different clouds; the
reference arm runs on rank 0 only.  (Each GPU machine here has one GPU, so the ranks are
replicas with no collective on the data path.)"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    dist = bench.dist_init(world, "gloo")
    t, u = bench.aggregate(10.0 + 5.0 * rank, 100.0 * (rank + 1), world)
    r, w, lr = bench.dist_env()
    ref = bench.reference_arm(bench.parse_args(["--impl", "reference", "--points", "1000", "--steps", "1",
                                                "--warmup", "0"]), dict(bench.WORKLOAD, points=1000)) \
        if rank == 1 else None
    out.put((rank, t, u, (r, w, lr), ref))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_aggregate_max_time_and_sum_of_units():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    by_rank = {g[0]: g for g in got}
    for rank in (0, 1):
        _, t, u, env, _ = by_rank[rank]
        assert t == 15.0 and u == 300.0  # max of 10 and 15 ms; 100 + 200 units
        assert env == (rank, 2, rank)
    assert by_rank[1][4] == 0  # the reference arm is rank 0's alone


def test_replicas_draw_different_clouds():
    sys.path.insert(0, ROOT)
    import synth

    a = synth.lidar_tile(2000, synth.CONFIG_SEED[2] + 0)
    b = synth.lidar_tile(2000, synth.CONFIG_SEED[2] + 1)
    assert a.shape == b.shape and not (a == b).all()
