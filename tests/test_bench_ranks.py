"""Multi-process host logic of the benchmark on CPU: two gloo ranks (replicas)
agree on the slowest rank's time and the whole-job rate; only rank 0 reports."""
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


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks("gloo")
    r.barrier()
    t = [0.25, 0.5][rank]                      # rank 1 is the slow one
    slowest = r.max(t)
    rate = r.whole_job_rate(1000.0, t)
    q.put((rank, r.world, slowest, rate))
    r.close()


def test_two_gloo_ranks_take_the_max_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, world, slowest, rate in res:
        assert world == 2
        assert slowest == 0.5
        assert rate == pytest.approx(2 * 1000.0 / 0.5)


def test_single_process_ranks_need_no_group():
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    r = bench.Ranks("gloo")
    assert r.world == 1 and r.rank == 0 and r.max(3.0) == 3.0
    assert r.whole_job_rate(10.0, 2.0) == 5.0
    r.close()
