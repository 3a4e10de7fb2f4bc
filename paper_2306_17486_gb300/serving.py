"""Batched mixed-size serving of Helmholtz solves on one GPU.

Requests arrive interleaved across grid sizes; each asks for the solutions of a batch of
right-hand sides (point sources) for its own slowness model.  Per grid size ("bucket")
the server keeps one problem handle, one network handle (grids up to the network's
limit) and one captured solver plan (helm_solver_plan_*: every restart cycle one CUDA
graph launch), on a CUDA stream of its own served by a host thread of its own, so the
buckets run concurrently on the device.  A request is served by
    helm_problem_update  (the bucket's problem, in place, for the request's model)
    helm_cnn_set_problem (the encoder on that model, once per request)
    copy of the right-hand sides from pinned host memory into the plan's buffer
    helm_solver_plan_solve
    copy of the solutions back into pinned host memory.
Latency is measured from the moment all requests are submitted (a burst in arrival
order) to each request's completion; the report gives p50 / p99 latency, the makespan
and the throughput in right-hand sides per second.  The same request stream served by
SL-multigrid-only plans is the reference the learned preconditioner is judged against.

    python -m paper_2306_17486_gb300.serving [--sizes 256,512,1024] [--requests 4]
        [--batch 8] [--mg-only]
"""
from __future__ import annotations

import argparse
import json
import os
import queue
import threading
import time

import numpy as np
import torch

from . import Cnn, Problem, SolverPlan, autotune, problem_update
from . import train as T

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "cnn_grf_multiscale.npz")
NET_MAX = 2304          # the network's largest grid (convolution windows within shared memory)


LEVELS = {288: 4, 576: 4, 1152: 5, 2304: 6}   # coarsest grids 36^2, 72^2, 72^2, 72^2


def bucket_config(n: int):
    """Grid of interior size n: absorbing layer max(16, n/16) cells per side (N = 288,
    576, 1152, 2304 for n = 256 ... 2048), the V-cycle depth of the benchmark workloads
    (other sizes: deepened until the coarsest grid is at most 72^2 or N cannot be halved
    again), iteration cap."""
    abl = max(16, n // 16)
    N = n + 2 * abl
    levels = LEVELS.get(N)
    if levels is None:
        # deepen while the coarsest grid is above 72^2 and the next level still divides N
        levels = 2
        while levels < 8 and (N >> (levels - 1)) > 72 and N % (1 << levels) == 0:
            levels += 1
    maxit = 2000 if N <= 600 else (4000 if N <= 1200 else 8000)
    return N, abl, levels, maxit


class Bucket:
    """One grid size: problem, optional network, captured plan, stream, worker thread."""

    def __init__(self, n: int, batch: int, use_net: bool, cnn_every: int, first_kappa: np.ndarray, device="cuda"):
        self.n = n
        self.N, self.abl, self.levels, self.maxit = bucket_config(n)
        self.batch = batch
        self.stream = torch.cuda.Stream(device=device)
        self.device = torch.device(device)
        self.use_net = use_net and self.N <= NET_MAX
        with torch.cuda.stream(self.stream):
            kt = torch.tensor(first_kappa, dtype=torch.float32, device=device)
            self.problem = Problem(kt, self.abl, self.omega_h(first_kappa), levels=self.levels)
            self.net = None
            if self.use_net:
                self.net = Cnn(skip_threshold=256, device=device)
                T.load_weights(self.net, WEIGHTS)
                self.net.set_problem(self.problem)
            self.plan = SolverPlan(self.problem, batch, cnn=self.net, restart=10, rtol=1e-6, maxit=self.maxit,
                                   warmup_iters=3, cnn_every=cnn_every, stream=self.stream)
        self.kdev = torch.empty((self.N, self.N), dtype=torch.float32, device=device)
        self.hb = torch.empty((batch, self.N, self.N), dtype=torch.complex64).pin_memory()
        self.hx = torch.empty((batch, self.N, self.N), dtype=torch.complex128).pin_memory()
        self.q: queue.Queue = queue.Queue()

    @staticmethod
    def omega_h(kappa: np.ndarray) -> float:
        return 2.0 * np.pi / (10.0 * float(kappa.max()))   # 10 points per wavelength at the largest kappa

    def serve(self, kappa: np.ndarray, b: np.ndarray):
        """Solve one request on the bucket's stream; returns the per-RHS statistics."""
        with torch.cuda.stream(self.stream):
            self.kdev.copy_(torch.from_numpy(kappa.astype(np.float32)), non_blocking=False)
            problem_update(self.problem, self.kdev, self.omega_h(kappa))
            if self.net is not None:
                self.net.set_problem(self.problem)
            self.hb.copy_(torch.from_numpy(b))
            self.plan.b.copy_(self.hb, non_blocking=True)
            st = self.plan.solve()
            self.hx.copy_(self.plan.x, non_blocking=True)
            self.stream.synchronize()
        return st

    def close(self):
        self.plan.close()
        if self.net is not None:
            self.net.close()
        self.problem.close()


def make_requests(sizes, per_size: int, batch: int, seed: int = 0):
    """Interleaved request stream: round robin over the sizes, each request its own
    layered+GRF slowness model and `batch` seeded point sources."""
    import synth
    reqs = []
    for k in range(per_size):
        for n in sizes:
            N, abl, _, _ = bucket_config(n)
            s = seed + 1000 * k + n
            kap = synth.layered_grf_kappa(n, abl, seed=s)
            b = synth.random_point_sources(N, abl, batch, seed=s + 1).astype(np.complex64)
            reqs.append({"id": len(reqs), "n": n, "kappa": kap, "b": b})
    return reqs


def run(sizes=(256, 512, 1024), per_size=4, batch=8, mg_only=False, cnn_every=3, seed=0, warm=True):
    """Serve the interleaved request stream; returns the report dict."""
    reqs = make_requests(sizes, per_size, batch, seed)
    first = {r["n"]: r["kappa"] for r in reversed(reqs)}
    autotune.apply(grids={(bucket_config(n)[0], batch) for n in sizes})   # before the plans are captured
    buckets = {n: Bucket(n, batch, not mg_only, cnn_every, first[n]) for n in sizes}
    if warm:   # one untimed request per bucket
        for n, bk in buckets.items():
            bk.serve(first[n], np.zeros((batch, bk.N, bk.N), dtype=np.complex64))
    torch.cuda.synchronize()
    done = {}
    errors = []

    def worker(bk: Bucket):
        while True:
            r = bk.q.get()
            if r is None:
                return
            try:
                st = bk.serve(r["kappa"], r["b"])
                done[r["id"]] = (time.perf_counter(), st)
            except Exception as exc:   # reported after the run
                errors.append(repr(exc))
                done[r["id"]] = (time.perf_counter(), None)

    threads = [threading.Thread(target=worker, args=(bk,), daemon=True) for bk in buckets.values()]
    for t in threads:
        t.start()
    t0 = time.perf_counter()
    for r in reqs:
        buckets[r["n"]].q.put(r)
    for bk in buckets.values():
        bk.q.put(None)
    for t in threads:
        t.join()
    makespan = time.perf_counter() - t0
    lat = np.array([done[r["id"]][0] - t0 for r in reqs]) * 1e3
    per_size = {}
    for n in sizes:
        sel = [i for i, r in enumerate(reqs) if r["n"] == n]
        sts = [done[reqs[i]["id"]][1] for i in sel]
        its = np.concatenate([s["iters"] for s in sts if s is not None]) if sts else np.zeros(0)
        conv = np.concatenate([s["status"] == 1 for s in sts if s is not None]) if sts else np.zeros(0)
        per_size[str(buckets[n].N)] = {"p50_ms": round(float(np.percentile(lat[sel], 50)), 2),
                                       "iterations_mean": round(float(its.mean()), 1) if its.size else None,
                                       "converged_frac": float(conv.mean()) if conv.size else None,
                                       "network": buckets[n].use_net}
    rep = {"method": "sl-mg only" if mg_only else f"cnn+sl-mg (network every {cnn_every} steps)",
           "grids": [buckets[n].N for n in sizes], "requests": len(reqs), "rhs_per_request": batch,
           "p50_ms": round(float(np.percentile(lat, 50)), 2), "p99_ms": round(float(np.percentile(lat, 99)), 2),
           "makespan_s": round(makespan, 3), "throughput_rhs_per_s": round(len(reqs) * batch / makespan, 2),
           "per_grid": per_size, "errors": errors}
    for bk in buckets.values():
        bk.close()
    return rep


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default="256,512,1024")
    ap.add_argument("--requests", type=int, default=4, help="requests per size")
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--cnn-every", type=int, default=3)
    ap.add_argument("--mg-only", action="store_true")
    a = ap.parse_args()
    sizes = tuple(int(v) for v in a.sizes.split(","))
    print(json.dumps(run(sizes, a.requests, a.batch, a.mg_only, a.cnn_every)))


if __name__ == "__main__":
    main()
