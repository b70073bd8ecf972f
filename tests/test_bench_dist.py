"""Host logic of the multi-GPU bench path on the CPU (gloo, world size 2).

bench.py shards independent right-hand sides over ranks (one seed per rank, no collective on the data
path) and reports the whole-job throughput with the time maximised over ranks; these are the pieces
that run on the host, exercised here with two gloo processes.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        seed = bench.rank_seed(r)
        mine = 1.0 + r  # rank-dependent elapsed time
        tmax = bench.reduce_max(mine)
        bench.barrier()
        value = bench.aggregate(10, ws, tmax)
        out.put((r, ws, seed, tmax, value))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_max_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ws0, s0, t0, v0), (r1, ws1, s1, t1, v1) = res
    assert (ws0, ws1) == (2, 2)
    assert s0 != s1  # independent right-hand sides per rank
    assert t0 == t1 == 2.0  # the slowest rank's time
    assert v0 == v1 == pytest.approx(10 * 2 / 2.0)


def test_single_process_defaults():
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.reduce_max(3.5) == 3.5
    assert bench.aggregate(120, 1, 0.5) == 240.0
    args = bench.parse_args([])
    assert args.gpus == 1 and args.warmup >= 3 and args.steps > 0
