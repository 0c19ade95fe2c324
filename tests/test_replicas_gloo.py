"""The multi-GPU path of bench.py is replicas only: every rank solves its own
copy of the workload, the ranks meet at a barrier, the job time is the
slowest rank's and the whole-job value counts all ranks' eigenpairs.  This
checks that host logic with two gloo ranks on the CPU (no GPU, no solve)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    r, w = bench.dist_init("gloo")
    ms = 1000.0 * (r + 1)  # rank 1 is the slow one
    bench.dist_barrier(w)
    mx = bench.dist_max(ms, w)
    out.put((r, w, mx, bench.job_value(w, 500, 1, mx)))
    import torch.distributed as dist

    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, mx, val in res:
        assert w == world
        assert mx == 2000.0  # max over ranks
        assert val == pytest.approx(2 * 500 / 2.0)  # 1000 eigenpairs in 2 s
