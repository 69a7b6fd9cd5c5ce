"""The N > 1 path of bench.py on CPU: two ranks joined over gloo (127.0.0.1).

The sweep of one chain runs on one GPU; with several GPUs bench.py runs
independent replicas, joined only by a barrier before and after the timed
region and a max over the ranks' times. This test runs those pieces (process
group set-up from the torchrun environment, barrier, max reduction, whole-job
throughput, rank-0-only reference arm) in two CPU processes.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup(None)
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    ms_max = bench.allreduce_max(ms, w)
    value = bench.job_value(3, ms_max, w)

    class Args:
        steps, warmup, chi, gpus = 1, 0, 8, world
    if rank != 0:
        assert bench.run_reference(Args, w, r) is None   # ranks > 0 do no work
    bench.barrier(w)
    out.put((rank, ms_max, value))
    dist.destroy_process_group()


def test_two_replicas_over_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value in res:
        assert ms_max == 150.0
        assert abs(value - 3 * 2 / 0.150) < 1e-9
