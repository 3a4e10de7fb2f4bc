"""Workloads for kernel profiling (ncu) and quick per-kernel timing: each case builds the
576^2 (512^2 interior + 32-cell absorbing layer) benchmark problem on slowness model 0,
runs `--warmup` untimed repetitions and `--reps` repetitions of one hot-path call, and
prints the library's per-kernel CUDA-event times for the repetitions.

    python -m paper_2306_17486_gb300.profile_case apply|vcycle|cnn|precond|solve [--batch B]
        [--reps R] [--warmup W] [--weights npz] [--maxit K] [--bc dirichlet|neumann|sommerfeld]
        [--explicit]

  apply    Helmholtz matvec y = h^2 A x on B random vectors
  vcycle   one SL V(1,1) cycle on B random residuals
  cnn      the network alone, e = s Net(r / s)
  precond  the composed preconditioner z = e + V(r - A e)
  solve    FGMRES(10) with the composed preconditioner (--mg-only: V-cycle alone) on B
           point sources, at most --maxit iterations
--bc selects the boundary condition of the problem; --explicit times the explicit U-Net
(the network without the implicit step, randomly initialised: its timing does not depend
on the weights).
"""
from __future__ import annotations

import argparse
import ctypes as C
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["apply", "vcycle", "cnn", "precond", "solve"])
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--weights", default=os.path.join(ROOT, "paper_2306_17486_gb300", "weights",
                                                      "cnn_grf_multiscale.npz"))
    ap.add_argument("--maxit", type=int, default=50)
    ap.add_argument("--mg-only", action="store_true")
    ap.add_argument("--bc", default="dirichlet", choices=["dirichlet", "neumann", "sommerfeld"])
    ap.add_argument("--explicit", action="store_true")
    a = ap.parse_args()
    sys.path.insert(0, ROOT)
    import synth
    from . import Cnn, Problem, fgmres_solve, helmholtz_apply, slmg_vcycle
    from . import train as T
    from ._lib import lib
    dev = "cuda"
    kap = synth.grf_kappa(512, 32, 8.0, seed=10)
    p = Problem(torch.tensor(kap, dtype=torch.float32, device=dev), 32, 2 * np.pi / 10 / float(kap.max()), levels=4,
                bc=a.bc)
    B = a.batch
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    r = torch.randn((B, 576, 576), dtype=torch.complex64, device=dev, generator=g)
    net = None
    if a.case in ("cnn", "precond") or (a.case == "solve" and not a.mg_only):
        net = Cnn(skip_threshold=256, explicit_unet=a.explicit)
        if a.explicit:
            net.load_dict(synth.random_params(T.init_spec(net), seed=0))
        else:
            T.load_weights(net, a.weights)
        net.set_problem(p)
    if a.case == "solve":
        b = torch.tensor(synth.random_point_sources(576, 32, B, seed=1000), dtype=torch.complex64, device=dev)

    def once():
        if a.case == "apply":
            helmholtz_apply(p, r)
        elif a.case == "vcycle":
            slmg_vcycle(p, r)
        elif a.case == "cnn":
            net.apply(p, r)
        elif a.case == "precond":
            net.precond(p, r)
        else:
            fgmres_solve(p, b, cnn=None if a.mg_only else net, restart=10, rtol=1e-6, maxit=a.maxit)

    for _ in range(a.warmup):
        once()
    torch.cuda.synchronize()
    L = lib()
    L.helm_profile_begin()
    for _ in range(a.reps):
        once()
    torch.cuda.synchronize()
    nk = C.c_int()
    L.helm_profile_end(C.byref(nk))
    rows = []
    for i in range(nk.value):
        nm, cnt, tot = C.c_char_p(), C.c_long(), C.c_double()
        L.helm_profile_read(i, C.byref(nm), C.byref(cnt), C.byref(tot))
        rows.append((tot.value / a.reps, cnt.value / a.reps, nm.value.decode()))
    rows.sort(reverse=True)
    total = sum(t for t, _, _ in rows)
    print(f"case {a.case}, batch {B}: {total:.3f} ms of kernel time per repetition")
    for t, n, name in rows:
        print(f"  {t:9.3f} ms  {n:7.1f} launches  {name}")


if __name__ == "__main__":
    main()
