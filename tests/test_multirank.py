"""The benchmark's multi-process path on CPU (gloo, world size 2): each rank
iterates its own replica, the job time is the maximum over ranks and the
whole-job value counts the points all ranks processed.  The path has no
data-path collective, so this is all the N > 1 logic there is."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    assert bench.dist_setup() == (ws, rank, rank)
    local_seconds = 2.0 if rank == 0 else 3.0  # rank 1 is the slowest
    value, t = bench.job_throughput(1000, 10, local_seconds, device="cpu")
    dist.barrier()
    q.put((rank, value, t))
    dist.destroy_process_group()


def test_job_throughput_max_over_two_gloo_ranks():
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
    for rank, value, t in res:
        assert t == pytest.approx(3.0)
        assert value == pytest.approx(1000 * 10 * 2 / 3.0)


def test_job_throughput_single_process():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    v, t = bench.job_throughput(500, 4, 2.0)
    assert (v, t) == (1000.0, 2.0)
