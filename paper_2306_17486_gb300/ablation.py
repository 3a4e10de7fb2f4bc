"""The comparison of Section 6: the implicit U-Net against the explicit U-Net (the same
encoder-solver network without the implicit step at the coarsest level), each followed
by the SL V-cycle as an FGMRES(10) preconditioner, beside the V-cycle alone.

Both networks start from the same initial parameters (the implicit kernels are the only
extra tensor, set to L + iI) and are trained by the same multiscale schedule on the same
Eq. 17 data stream: one seed fixes the slowness pool, the input vectors and the
iteration counts, and the pairs come from the plain solver, so they do not depend on the
network.  Each test grid is one seeded GRF slowness model with `--rhs` point sources,
solved to a 1e-6 relative residual.

    python -m paper_2306_17486_gb300.ablation [--steps S] [--sizes 128:16:3,256:32:3]
        [--test 288:16:4,576:32:4,1152:64:5] [--rhs R] [--cnn-every K] [--maxit M] [--out file.json]

The JSON written to --out is rewritten after every phase, so an interrupted run keeps
what it measured.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sizes(text: str):
    return tuple(tuple(int(v) for v in t.split(":")) for t in text.split(","))


def solve_row(helm, p, b, net, cnn_every: int, maxit: int = 2000) -> dict:
    """One FGMRES(10) solve of the batch b; iteration statistics and ms per RHS."""
    helm.fgmres_solve(p, b, cnn=net, restart=10, rtol=1e-6, maxit=5, cnn_every=cnn_every)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, st = helm.fgmres_solve(p, b, cnn=net, restart=10, rtol=1e-6, maxit=maxit, cnn_every=cnn_every)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    it = st["iters"].astype(np.float64)
    return {"iterations_mean": float(it.mean()), "iterations_max": int(it.max()),
            "converged_frac": float((st["status"] == 1).mean()), "ms_per_rhs": 1e3 * dt / b.shape[0]}


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--steps", type=int, default=2000, help="training steps of each network")
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--sizes", default="128:16:3,256:32:3", help="training grids N_total:abl:levels")
    ap.add_argument("--test", default="288:16:4,576:32:4", help="test grids N_total:abl:levels")
    ap.add_argument("--rhs", type=int, default=16)
    ap.add_argument("--cnn-every", type=int, default=1)
    ap.add_argument("--maxit", type=int, default=2000, help="iteration cap of the test solves")
    ap.add_argument("--skip-threshold", type=int, default=256)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    sys.path.insert(0, ROOT)
    import synth

    import paper_2306_17486_gb300 as helm
    from . import train as T

    res = {"what": "implicit vs explicit U-Net (Section 6), equal training", "steps": a.steps, "batch": a.batch,
           "train_sizes": a.sizes, "rhs": a.rhs, "cnn_every": a.cnn_every, "maxit": a.maxit, "seed": a.seed,
           "train": {}, "test": []}

    def dump():
        if a.out:
            with open(a.out, "w") as f:
                json.dump(res, f, indent=1)

    nets = {}
    for name, explicit in (("explicit", True), ("implicit", False)):
        net = helm.Cnn(skip_threshold=a.skip_threshold, explicit_unet=explicit)
        net.load_dict(synth.random_params(T.init_spec(net), seed=a.seed))
        tr = T.Trainer(net, sizes=_sizes(a.sizes), batch=a.batch, steps=a.steps, seed=a.seed)
        t0 = time.time()
        hist = tr.run(a.steps, log=None)
        torch.cuda.synchronize()
        res["train"][name] = {"params": net.nparams, "seconds": time.time() - t0,
                              "final_loss": hist[-1][2] if hist else None}
        print(f"trained {name}: {net.nparams} parameters, {a.steps} steps, {time.time() - t0:.1f} s, "
              f"loss {res['train'][name]['final_loss']}", flush=True)
        nets[name] = net
        dump()
    for N, abl, lv in _sizes(a.test):
        kap = synth.grf_kappa(N - 2 * abl, abl, 8.0, seed=10)
        p = helm.Problem(torch.tensor(kap, dtype=torch.float32, device="cuda"), abl,
                         2 * np.pi / (10.0 * float(kap.max())), levels=lv)
        b = torch.tensor(synth.random_point_sources(N, abl, a.rhs, seed=1000), dtype=torch.complex64, device="cuda")
        row = {"grid": N, "abl": abl, "levels": lv, "mg_only": solve_row(helm, p, b, None, a.cnn_every, a.maxit)}
        for name, net in nets.items():
            net.set_problem(p)
            row[name] = solve_row(helm, p, b, net, a.cnn_every, a.maxit)
        res["test"].append(row)
        print(json.dumps(row), flush=True)
        dump()


if __name__ == "__main__":
    main()
