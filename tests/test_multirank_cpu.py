"""The multi-rank bench path (one replica per rank, barrier, max over ranks) on
world_size 2 with the gloo backend on CPU processes."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), BENCH_BACKEND="gloo")
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import bench
    w, r, _ = bench.dist_setup(world)
    bench.barrier(w)
    ms = 100.0 * (r + 1)                      # rank 1 is the slow one
    ms_max = bench.max_over_ranks(w, ms, torch.device("cpu"))
    q.put((r, w, ms_max, bench.job_throughput(w, 50, ms_max)))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
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
    for r, w, ms_max, value in res:
        assert w == 2 and ms_max == pytest.approx(200.0)
        assert value == pytest.approx(2 * 50 / 0.2)
