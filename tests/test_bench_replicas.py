"""bench.py's multi-GPU mode runs independent replicas (one process per GPU, no collective on
the data path): a timed region lasts as long as its slowest rank, and the whole-job rate
counts every rank's units.  The reduction is checked with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ws_env, rank_env, _ = bench.dist_env()
        times = [1.0 + rank, 10.0 - rank, 3.0]          # per-rank timings of three regions
        got = bench.max_over_ranks(times, ws_env, device="cpu")
        rate = bench.replica_rate(ws_env, 20, got[0])
        q.put((rank_env, got, rate))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = {}
        for _ in range(2):
            r, got, rate = q.get(timeout=180)
            res[r] = (got, rate)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    # every rank sees the slowest rank's time of each region, and 2 x 20 units in 2 ms
    assert res[0] == res[1] == ([2.0, 10.0, 3.0], 20000.0)


def test_single_rank_is_the_identity():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
    assert bench.replica_rate(1, 20, 1000.0) == 20.0
    assert bench.replica_rate(4, 20, 1000.0) == 80.0
