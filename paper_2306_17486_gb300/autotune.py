"""Launch-shape autotuner for the network's convolution and inverted-bottleneck kernels.

The launchers pick their work-unit shapes by heuristics (output rows per convolution
segment from the shared-memory budget; rows per inverted-bottleneck strip unit from a
wave-balance model).  For one grid size N and batch B this module times the network
application e = s Net(r / s) with CUDA events and, height by height of the U-Net's
levels, tries the candidates of each knob, keeping a value only where it beats the
current shape by more than `min_gain`.  The result goes to the library's tuning table
(helm_tune_set, keyed by knob, layer height and batch) and to a JSON file that
`apply()` loads into the table of another process (the serving buckets, the benchmark).

    python -m paper_2306_17486_gb300.autotune --grids 576:64,288:8,576:8,1152:8 \
        [--out paper_2306_17486_gb300/tuning/launch_shapes.json]
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np
import torch

from . import Cnn, Problem, tune_set
from . import train as T

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "cnn_grf_multiscale.npz")
DEFAULT_PATH = os.path.join(HERE, "tuning", "launch_shapes.json")

CANDIDATES = {"conv_rows": (2, 4, 8, 12, 16, 24, 32), "ib_sh": (4, 8, 12, 16, 20, 24, 32, 48)}


def _time_ms(fn, reps: int) -> float:
    """Median CUDA-event time of fn() on the current stream, after two warm-up calls."""
    for _ in range(2):
        fn()
    st = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def level_heights(N: int, levels: int = 6):
    """Heights of the network's levels on an N x N grid (each level halves the grid)."""
    hs = []
    for lv in range(levels):
        if N % (1 << lv) or (N >> lv) < 8:
            break
        hs.append(N >> lv)
    return hs


def tune_grid(N: int, abl: int, batch: int, seed: int = 0, reps: int = 7, min_gain: float = 0.02, knobs=None):
    """Tune the knobs for the network on an N x N grid and `batch` right-hand sides.
    Returns {"N", "batch", "entries": [(knob, height, value)], "ms_heuristic", "ms_tuned"}
    and leaves the chosen entries in the library's table."""
    import synth
    knobs = knobs or tuple(CANDIDATES)
    n = N - 2 * abl
    kap = torch.tensor(synth.layered_grf_kappa(n, abl, seed=seed), dtype=torch.float32, device="cuda")
    p = Problem(kap, abl, 2 * np.pi / 10 / float(kap.max()), levels=2)
    net = Cnn(skip_threshold=256)
    T.load_weights(net, WEIGHTS)
    net.set_problem(p)
    g = torch.Generator().manual_seed(seed + 1)
    r = torch.complex(torch.randn(batch, N, N, generator=g), torch.randn(batch, N, N, generator=g))
    r = r.to(torch.complex64).cuda()
    ws = p.workspace(batch, 10, net)

    def run():
        net.apply(p, r, ws=ws)

    heights = level_heights(N)
    for knob in knobs:
        for h in heights:
            tune_set(knob, h, batch, 0)
    ms0 = _time_ms(run, reps)
    best_ms = ms0
    entries = []
    for knob in knobs:
        for h in heights:
            keep, keep_ms = 0, best_ms
            for c in CANDIDATES[knob]:
                tune_set(knob, h, batch, c)
                t = _time_ms(run, reps)
                if t < keep_ms * (1 - min_gain):
                    keep, keep_ms = c, t
            tune_set(knob, h, batch, keep)
            if keep:
                entries.append((knob, h, keep))
                best_ms = keep_ms
    ms1 = _time_ms(run, 3 * reps)
    net.close()
    p.close()
    return {"N": N, "batch": batch, "entries": entries, "ms_heuristic": round(ms0, 4), "ms_tuned": round(ms1, 4)}


def save(results, path: str = DEFAULT_PATH):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    doc = {"device": torch.cuda.get_device_name(), "what": "network application e = s Net(r/s), CUDA-event median",
           "grids": [{"N": r["N"], "batch": r["batch"], "ms_heuristic": r["ms_heuristic"], "ms_tuned": r["ms_tuned"],
                      "entries": [{"knob": k, "height": h, "value": v} for k, h, v in r["entries"]]}
                     for r in results]}
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")


def apply(path: str = DEFAULT_PATH, grids=None) -> int:
    """Load tuned entries into the library's table (only the (N, batch) pairs in `grids`
    when given).  Returns the number of entries set; a missing file sets none."""
    if not os.path.exists(path):
        return 0
    with open(path) as f:
        doc = json.load(f)
    count = 0
    for gr in doc.get("grids", []):
        if grids is not None and (gr["N"], gr["batch"]) not in grids:
            continue
        for e in gr["entries"]:
            tune_set(e["knob"], e["height"], gr["batch"], e["value"])
            count += 1
    return count


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grids", default="576:64", help="N:batch pairs (N = interior + 2 * max(16, interior/16))")
    ap.add_argument("--reps", type=int, default=7)
    ap.add_argument("--out", default=DEFAULT_PATH)
    a = ap.parse_args()
    results = []
    for item in a.grids.split(","):
        N, B = (int(v) for v in item.split(":"))
        abl = max(16, N // 18)
        results.append(tune_grid(N, abl, B, reps=a.reps))
        print(json.dumps(results[-1]), flush=True)
    save(results, a.out)


if __name__ == "__main__":
    main()
