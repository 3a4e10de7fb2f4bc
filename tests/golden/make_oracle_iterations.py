"""Writes oracle_iterations_576.json: the FP64 oracle's own FGMRES(10) iteration counts
to a 1e-6 relative residual on the 576^2 benchmark workload (512^2 interior plus a
32-cell absorbing layer, GRF slowness seed 10, point sources seed 1000, 4-level V-cycle
with the coarsest GMRES(10)-Jacobi solve), for the first right-hand sides of the first
slowness model: with the SL V-cycle alone, and (--cnn) with the composed preconditioner
of the committed trained weights after a 3-iteration V-cycle warm-up cycle.  Calls only
oracle/ and synth/ (the weights file is read as plain arrays).

    python tests/golden/make_oracle_iterations.py [n_rhs]          # V-cycle only
    python tests/golden/make_oracle_iterations.py --cnn [n_rhs]    # CNN + V-cycle
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import fgmres as ofg  # noqa: E402
from oracle import helmholtz as ohz  # noqa: E402
from oracle import multigrid as omg  # noqa: E402

N_INT, ABL, LEVELS, RESTART, RTOL, MAXIT = 512, 32, 4, 10, 1e-6, 2000


WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(HERE)), "paper_2306_17486_gb300", "weights",
                       "cnn_grf_multiscale.npz")


def _network():
    from oracle import cnn as ocnn
    d = np.load(WEIGHTS)
    flat = d["params"].astype(np.float64)
    P, off = {}, 0
    for name, shape, *_ in ocnn.param_spec(16):
        n = int(np.prod(shape))
        P[name] = flat[off:off + n].reshape(shape)
        off += n
    assert off == flat.size
    run = d["running"].astype(np.float64)
    R, off = {}, 0
    for name, c in ocnn.bn_names(16):
        R[name] = (run[off:off + c], run[off + c:off + 2 * c])
        off += 2 * c
    return ocnn.Network(P, R, c0=16)


def main_cnn(n_rhs: int = 1):
    from oracle import cnn as ocnn
    from oracle import training as otr
    kappa = synth.grf_kappa(N_INT, ABL, 8.0, seed=10)
    b = synth.random_point_sources(N_INT + 2 * ABL, ABL, 64, seed=1000)
    p = ohz.Problem(kappa, ABL)
    mg = omg.SLMultigrid(p, LEVELS)
    net = _network()
    M = otr.composed_preconditioner(p, net, ocnn.kappa_features(p.kappa, p.gamma), mg)
    out = []
    for i in range(n_rhs):
        t0 = time.perf_counter()
        bi = b[i].astype(np.complex128)
        x, r1 = ofg.fgmres(p.A, bi, np.zeros_like(bi), mg, 3, RTOL, 3)          # warm-up cycle
        x, r2 = ofg.fgmres(p.A, bi, x, M, RESTART, RTOL, MAXIT - r1.iters, bnorm=np.linalg.norm(bi))
        rel = float(np.linalg.norm(bi - p.A(x)) / np.linalg.norm(bi))
        out.append({"rhs": i, "iterations": int(r1.iters + r2.iters), "true_rel_res": rel,
                    "seconds": round(time.perf_counter() - t0, 1)})
        print(out[-1], flush=True)
    path = os.path.join(HERE, "oracle_iterations_576.json")
    doc = json.load(open(path)) if os.path.exists(path) else {}
    doc["cnn_mg"] = {"what": "oracle FGMRES(10) with the composed CNN + V-cycle preconditioner (committed weights "
                             "cnn_grf_multiscale.npz), 3 V-cycle warm-up iterations, to 1e-6",
                     "results": out, "mean_iterations": float(np.mean([o["iterations"] for o in out]))}
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)


def main(n_rhs: int = 4):
    kappa = synth.grf_kappa(N_INT, ABL, 8.0, seed=10)
    b = synth.random_point_sources(N_INT + 2 * ABL, ABL, 64, seed=1000)
    p = ohz.Problem(kappa, ABL)
    mg = omg.SLMultigrid(p, LEVELS)
    out = []
    for i in range(n_rhs):
        t0 = time.perf_counter()
        bi = b[i].astype(np.complex128)
        x, res = ofg.fgmres(p.A, bi, np.zeros_like(bi), mg, RESTART, RTOL, MAXIT)
        rel = float(np.linalg.norm(bi - p.A(x)) / np.linalg.norm(bi))
        out.append({"rhs": i, "iterations": int(res.iters), "true_rel_res": rel,
                    "seconds": round(time.perf_counter() - t0, 1)})
        print(out[-1], flush=True)
    path = os.path.join(HERE, "oracle_iterations_576.json")
    old = json.load(open(path)) if os.path.exists(path) else {}
    doc = {"what": "oracle SL-MG FGMRES(10) iterations to 1e-6 on the 576^2 benchmark workload",
           "kappa": "synth.grf_kappa(512, 32, 8.0, seed=10)",
           "rhs": "synth.random_point_sources(576, 32, 64, seed=1000)[i]",
           "solver": {"restart": RESTART, "rtol": RTOL, "maxit": MAXIT, "levels": LEVELS},
           "results": out,
           "mean_iterations": float(np.mean([o["iterations"] for o in out]))}
    if "cnn_mg" in old:
        doc["cnn_mg"] = old["cnn_mg"]
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if a != "--cnn"]
    if "--cnn" in sys.argv:
        main_cnn(int(args[0]) if args else 1)
    else:
        main(int(args[0]) if args else 4)
