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


def test_reference_arm_runs_on_rank_zero_only():
    """`bench.py --impl reference` under a two-rank launch: rank 1 does no work and exits
    0, rank 0 times the oracle and prints one JSON line with the reference-arm keys."""
    import json
    import subprocess
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0"]
    base = dict(os.environ, WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", OMP_NUM_THREADS="2")
    r1 = subprocess.run(cmd, env=dict(base, RANK="1", LOCAL_RANK="1"), capture_output=True, text=True, timeout=300)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = subprocess.run(cmd, env=dict(base, RANK="0", LOCAL_RANK="0"), capture_output=True, text=True, timeout=600)
    assert r0.returncode == 0, r0.stderr[-2000:]
    lines = [l for l in r0.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["higher_is_better"] is False
    assert d["unit"] == "ms/RHS" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 2
    assert d["e2e"] == {"value": d["value"], "unit": "ms/RHS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"]
