"""Writes oracle_iterations_576.json: the FP64 oracle's own FGMRES(10) + SL V-cycle
iteration counts to a 1e-6 relative residual on the 576^2 benchmark workload (512^2
interior plus a 32-cell absorbing layer, GRF slowness seed 10, point sources seed 1000,
4-level V-cycle with the coarsest GMRES(10)-Jacobi solve), for the first right-hand
sides of the first slowness model.  Calls only oracle/ and synth/.

    python tests/golden/make_oracle_iterations.py [n_rhs]
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
    doc = {"what": "oracle SL-MG FGMRES(10) iterations to 1e-6 on the 576^2 benchmark workload",
           "kappa": "synth.grf_kappa(512, 32, 8.0, seed=10)",
           "rhs": "synth.random_point_sources(576, 32, 64, seed=1000)[i]",
           "solver": {"restart": RESTART, "rtol": RTOL, "maxit": MAXIT, "levels": LEVELS},
           "results": out,
           "mean_iterations": float(np.mean([o["iterations"] for o in out]))}
    with open(os.path.join(HERE, "oracle_iterations_576.json"), "w") as f:
        json.dump(doc, f, indent=1)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 4)
