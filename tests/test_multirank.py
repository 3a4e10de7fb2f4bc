"""Host logic of the multi-GPU benchmark path on CPU (world size 2, gloo, 127.0.0.1):
replicas only, so each rank's slowness models and right-hand sides must be disjoint from
every other rank's, and the reported time is the maximum over ranks."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = bench.job_seeds(rank)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    t = bench.max_over_ranks(10.0 * (rank + 1), dist)
    if rank == 0:
        out.put((gathered, t))
    dist.destroy_process_group()


def test_two_ranks_disjoint_work_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    import socket
    with socket.socket() as sk:   # a port the OS reports free on 127.0.0.1
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    kap = [k for seeds in gathered for k, _ in seeds]
    rhs = [r for seeds in gathered for _, r in seeds]
    assert len(set(kap)) == len(kap) and len(set(rhs)) == len(rhs)
    assert t == 20.0
