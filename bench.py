"""Benchmark: ms per right-hand side to a 1e-6 relative residual, learned CNN + SL-MG
vs SL-MG-only preconditioned FGMRES, on one GB300 (or N replicas).

Workload (one "step"): a 512 x 512 grid plus a 32-cell absorbing layer (576^2 nodes),
4 seeded Gaussian-random-field slowness models in [0.25, 1], 64 point-source
right-hand sides per model solved in one batched call, FGMRES(10), 4-level V-cycle,
relative residual 1e-6 (true FP64 residual).  Inputs are generated once and resident
in HBM before timing; the Krylov basis (11 x 64 x 576^2 complex64 = 1.9 GB per model)
is far larger than L2, so no flush is needed between steps.

The same line carries `workload_1152`: the 1024^2 grid (plus a 64-cell layer, 1152^2
nodes, 5-level V-cycle), 2 slowness models x 16 point sources, each arm timed once; and
`serving`: p50/p99 latency of a burst of mixed-size requests (288^2, 576^2, 1152^2
nodes, 8 right-hand sides each) served by captured solver plans, with and without the
network; and `ood_shapes`: the trained network against SL-MG alone on the rectangular
out-of-distribution shapes of Section 5.1 (512 x 1024 and 352 x 800 interiors, 8 point
sources each); and `workload_2176`: the 2048^2 interior (2176^2 nodes, 6-level V-cycle),
one model x 8 point sources, the network against SL-MG alone.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--skip-1152]
        [--skip-serving] [--skip-ood] [--skip-2176]
        (N > 1: launched by torchrun, one replica per GPU, independent models per rank)
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms per RHS to 1e-6 rel. residual, CNN+MG vs MG-only preconditioned FGMRES"
N_INT, ABL, LEVELS = 512, 32, 4
N_MODELS, N_RHS, RESTART, RTOL, MAXIT = 4, 64, 10, 1e-6, 2000
# the composed CNN + V-cycle preconditioner on every CNN_EVERY-th Arnoldi step, the
# V-cycle alone on the others (flexible GMRES admits a different preconditioner per
# step); 1 is the paper's schedule, reported beside the headline
CNN_EVERY = 3
WORKLOAD = "helmholtz-576sq-4kappa-x64rhs-fgmres10"


def job_seeds(rank: int):
    """Replicas only: rank r solves its own N_MODELS slowness models with their own
    right-hand sides; (kappa seed, right-hand-side seed) per model, disjoint across ranks."""
    return [(10 + N_MODELS * rank + k, 1000 + N_MODELS * rank + k) for k in range(N_MODELS)]


def max_over_ranks(ms: float, dist, device=None) -> float:
    """The job's time is the slowest rank's (all ranks start after one barrier)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _kappas(rank: int):
    import synth
    return [synth.grf_kappa(N_INT, ABL, 8.0, seed=ks) for ks, _ in job_seeds(rank)]


def _rhs(rank: int, k: int):
    import synth
    return synth.random_point_sources(N_INT + 2 * ABL, ABL, N_RHS, seed=job_seeds(rank)[k][1])


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


# DRAM bytes per RHS of one application of a kernel family (all its launches), measured
# by ncu on captures at the bench shape (64 RHS x 576^2, tensors larger than the 129 MB
# L2): the matvec (one launch), the V-cycle legs (three launches each) and the network's
# families (dram__bytes_read.sum + dram__bytes_write.sum over one application).  A kernel
# changed since its capture is removed from this table.
NCU_TRAFFIC_PER_RHS = {"k_apply": 298.29e6 / 64, "k_resid_restrict": 252.9e6 / 64, "k_prolong_smooth": 417.2e6 / 64,
                       "k_conv_tc": 2033.9e6 / 64, "k_ib_strip": 414.2e6 / 64, "k_ib_fused": 42.7e6 / 64,
                       "k_proj_prolong": 296.2e6 / 64}

# FP32 lane peak for kernels bound by plain arithmetic: 152 SMs x 128 FP32 lanes x 2 FLOP
# (fused multiply-add) x 2.07 GHz
FP32_LANE_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def _net_layer_bytes(I: int, B: int):
    """Algorithmic bytes of one network application at grid I (solver only; the encodings
    are read once per launch from L2 and not counted): every activation read once and
    written once, BF16 NHWC.  Returns {kernel family: bytes}."""
    h = I // 2
    px = lambda n: n * n * B
    ib_strip = 4 * 16 * px(h) + 4 * 32 * px(h // 2)                            # read x, write y
    ib_fused = 4 * 64 * px(h // 4)
    conv = 0
    conv += (2 * 2 + 2 * 16) * px(h)                                             # l1: 2 -> 16
    conv += 2 * 16 * px(h) + 2 * 32 * px(h // 2)                                 # l2: s2 16 -> 32
    conv += 2 * 32 * px(h // 2) + 2 * 64 * px(h // 4)                            # l3: s2 32 -> 64
    conv += 2 * 64 * px(h // 4) + 2 * 64 * px(h // 8) + 2 * (2 * 64 * 2) * px(h // 8)   # l4: 3 convs
    for c_in, c_out, n in ((64, 64, h // 4), (64, 32, h // 2), (32, 16, h)):     # up modules
        conv += 2 * c_in * px(n // 2) + 2 * c_out * px(n)                        # transposed s2
        conv += 10 * c_out * px(n)                                               # conv1, conv2 (+ skip read)
    proj = 2 * 16 * px(h) + 8 * px(I)
    return {"k_ib_strip": ib_strip, "k_ib_fused": ib_fused, "k_conv_tc": conv, "k_proj_prolong": proj}


def _implicit_flops(I: int, B: int, C: int = 64):
    """Algorithmic FLOPs of one implicit layer (Eq. 14) as FFTs: per (sample, complex
    channel) 6m transforms of length n = 2m (m row and 2m column forward/inverse, m row
    inverse) at the conventional 5 n log2 n real FLOPs each, plus the product with G_hat
    (6 FLOPs per spectral point)."""
    m = I // 16
    n = 2 * m
    return B * (C // 2) * (6 * m * 5 * n * np.log2(n) + 6 * n * n)


def _vcycle_bytes(N: int, levels: int, B: int):
    """Algorithmic bytes of one V-cycle (complex64): level l down-leg reads r_l, writes the
    coarse residual (1/4 size); up-leg reads r_l and the coarse correction, writes z_l."""
    down = up = 0
    for l in range(levels - 1):
        n = (N >> l) ** 2 * B
        down += 8 * n + 2 * n
        up += 8 * n + 2 * n + 8 * n
    return {"k_resid_restrict": down, "k_prolong_smooth": up}


# The 1024^2 workload: 1024^2 interior + 64-cell absorbing layer = 1152^2 nodes, 5-level
# V-cycle (coarsest 72^2), two seeded GRF slowness models x 16 point sources, maxit 4000
# (SL-MG alone needs more than the paper's 2000 here)
N1K_INT, N1K_ABL, N1K_LEVELS, N1K_MODELS, N1K_RHS, N1K_MAXIT = 1024, 64, 5, 2, 16, 4000


def run_1152(helm, net, dev, rank: int):
    """ms per RHS to 1e-6 on the 1152^2 workload: SL-MG alone, CNN+SL-MG with the network on
    every CNN_EVERY-th step, and the paper's schedule (every step); one timed pass of all
    right-hand sides per arm after an untimed warm-up solve, inputs resident in HBM."""
    import torch
    import synth
    probs, bs = [], []
    for k in range(N1K_MODELS):
        kap = synth.grf_kappa(N1K_INT, N1K_ABL, 8.0, seed=20 + N1K_MODELS * rank + k)
        oh = 2.0 * np.pi / (10.0 * float(kap.max()))
        probs.append(helm.Problem(torch.tensor(kap, dtype=torch.float32, device=dev), N1K_ABL, oh, levels=N1K_LEVELS))
        bs.append(torch.tensor(synth.random_point_sources(N1K_INT + 2 * N1K_ABL, N1K_ABL, N1K_RHS,
                                                          seed=2000 + N1K_MODELS * rank + k),
                               dtype=torch.complex64, device=dev))
    N = N1K_INT + 2 * N1K_ABL
    xs = [torch.zeros((N1K_RHS, N, N), dtype=torch.complex128, device=dev) for _ in range(N1K_MODELS)]
    for p in probs:
        p.workspace(N1K_RHS, RESTART, net)

    def arm(cnn, every, maxit=N1K_MAXIT):
        stats = []
        for k in range(N1K_MODELS):
            xs[k].zero_()
            if cnn:
                net.set_problem(probs[k])
            _, st = helm.fgmres_solve(probs[k], bs[k], xs[k], cnn=net if cnn else None, restart=RESTART, rtol=RTOL,
                                      maxit=maxit, warmup_iters=3, cnn_every=every)
            stats.append(st)
        return np.concatenate(stats)

    arm(False, 1, 30)
    arm(True, CNN_EVERY, 30)
    torch.cuda.synchronize()
    out = {"workload": "helmholtz-1152sq-2kappa-x16rhs-fgmres10", "grid": N, "interior": N1K_INT, "abl": N1K_ABL,
           "mg_levels": N1K_LEVELS, "kappa_models": N1K_MODELS, "rhs_per_model": N1K_RHS, "maxit": N1K_MAXIT}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, cnn, every in (("value", True, CNN_EVERY), ("mg_only", False, 1), ("paper_schedule", True, 1)):
        torch.cuda.synchronize()
        e0.record()
        st = arm(cnn, every)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / (N1K_MODELS * N1K_RHS)
        rec = {"ms_per_rhs": round(ms, 3), "iterations_mean": round(float(st["iters"].mean()), 1),
               "converged_frac": float(np.mean(st["status"] == 1)), "max_true_rel_res": float(st["rel_res_true"].max())}
        out[name] = rec
    out["speedup_vs_mg_only"] = round(out["mg_only"]["ms_per_rhs"] / out["value"]["ms_per_rhs"], 3)
    out["paper_schedule_speedup_vs_mg_only"] = round(out["mg_only"]["ms_per_rhs"] / out["paper_schedule"]["ms_per_rhs"],
                                                     3)
    return out


# The out-of-distribution grid shapes of Section 5.1 (512 x 1024 and 352 x 800 interiors,
# rows x columns) with a 32-cell absorbing layer: synthetic stand-ins for its models
# (a layered + GRF field and a salt body), one model and OOD_RHS point sources each
OOD_SHAPES = ((512, 1024, "layered_grf"), (352, 800, "salt"))
OOD_ABL, OOD_LEVELS, OOD_RHS = 32, 4, 8


# The 2048^2 interior (+ 64-cell layer = 2176^2 nodes, 6-level V-cycle, coarsest 68^2):
# one GRF model x 8 point sources; the network's coarsest map (136^2) takes the
# three-pass implicit layer
N2K_INT, N2K_ABL, N2K_LEVELS, N2K_RHS, N2K_MAXIT = 2048, 64, 6, 8, 8000


def run_2176(helm, net, dev, rank: int):
    """ms per RHS and iterations to 1e-6 on the 2176^2 grid: the network on every
    CNN_EVERY-th step against SL-MG alone, one timed pass per arm after an untimed
    warm-up solve, inputs resident in HBM."""
    import torch
    import synth
    N = N2K_INT + 2 * N2K_ABL
    kap = synth.grf_kappa(N2K_INT, N2K_ABL, 8.0, seed=60 + rank)
    oh = 2.0 * np.pi / (10.0 * float(kap.max()))
    p = helm.Problem(torch.tensor(kap, dtype=torch.float32, device=dev), N2K_ABL, oh, levels=N2K_LEVELS)
    b = torch.tensor(synth.random_point_sources(N, N2K_ABL, N2K_RHS, seed=6000 + rank), dtype=torch.complex64,
                     device=dev)
    x = torch.zeros(b.shape, dtype=torch.complex128, device=dev)
    p.workspace(N2K_RHS, RESTART, net)
    net.set_problem(p)
    out = {"workload": "helmholtz-2176sq-1kappa-x8rhs-fgmres10", "grid": N, "interior": N2K_INT, "abl": N2K_ABL,
           "mg_levels": N2K_LEVELS, "rhs": N2K_RHS, "maxit": N2K_MAXIT}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, cnn in (("value", True), ("mg_only", False)):
        helm.fgmres_solve(p, b, x, cnn=net if cnn else None, restart=RESTART, rtol=RTOL, maxit=30, warmup_iters=3,
                          cnn_every=CNN_EVERY)
        x.zero_()
        torch.cuda.synchronize()
        e0.record()
        _, st = helm.fgmres_solve(p, b, x, cnn=net if cnn else None, restart=RESTART, rtol=RTOL, maxit=N2K_MAXIT,
                                  warmup_iters=3, cnn_every=CNN_EVERY)
        e1.record()
        torch.cuda.synchronize()
        out[name] = {"ms_per_rhs": round(e0.elapsed_time(e1) / N2K_RHS, 3),
                     "iterations_mean": round(float(st["iters"].mean()), 1),
                     "converged_frac": float(np.mean(st["status"] == 1)),
                     "max_true_rel_res": float(st["rel_res_true"].max())}
    out["speedup_vs_mg_only"] = round(out["mg_only"]["ms_per_rhs"] / out["value"]["ms_per_rhs"], 3)
    del p
    return out


def run_ood(helm, net, dev, rank: int):
    """ms per RHS and iterations to 1e-6 on the rectangular out-of-distribution shapes:
    the trained network (on every CNN_EVERY-th step) against SL-MG alone; one timed pass
    per arm after an untimed warm-up solve, inputs resident in HBM."""
    import torch
    import synth
    out = {"abl": OOD_ABL, "mg_levels": OOD_LEVELS, "rhs_per_model": OOD_RHS, "grids": []}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k, (h, w, kind) in enumerate(OOD_SHAPES):
        kap = synth.rect_kappa(h, w, OOD_ABL, seed=40 + 2 * rank + k, kind=kind)
        oh = 2.0 * np.pi / (10.0 * float(kap.max()))
        p = helm.Problem(torch.tensor(kap, dtype=torch.float32, device=dev), OOD_ABL, oh, levels=OOD_LEVELS)
        b = torch.tensor(synth.rect_point_sources(h, w, OOD_ABL, OOD_RHS, seed=4000 + 2 * rank + k),
                         dtype=torch.complex64, device=dev)
        x = torch.zeros(b.shape, dtype=torch.complex128, device=dev)
        p.workspace(OOD_RHS, RESTART, net)
        net.set_problem(p)
        rec = {"grid": [h + 2 * OOD_ABL, w + 2 * OOD_ABL], "interior": [h, w], "model": kind}
        for name, cnn in (("cnn_mg", True), ("mg_only", False)):
            helm.fgmres_solve(p, b, x, cnn=net if cnn else None, restart=RESTART, rtol=RTOL, maxit=30,
                              warmup_iters=3, cnn_every=CNN_EVERY)
            x.zero_()
            torch.cuda.synchronize()
            e0.record()
            _, st = helm.fgmres_solve(p, b, x, cnn=net if cnn else None, restart=RESTART, rtol=RTOL, maxit=MAXIT,
                                      warmup_iters=3, cnn_every=CNN_EVERY)
            e1.record()
            torch.cuda.synchronize()
            rec[name] = {"ms_per_rhs": round(e0.elapsed_time(e1) / OOD_RHS, 3),
                         "iterations_mean": round(float(st["iters"].mean()), 1),
                         "converged_frac": float(np.mean(st["status"] == 1)),
                         "max_true_rel_res": float(st["rel_res_true"].max())}
        rec["speedup_vs_mg_only"] = round(rec["mg_only"]["ms_per_rhs"] / rec["cnn_mg"]["ms_per_rhs"], 3)
        out["grids"].append(rec)
        del p
    return out


COMPARISON_KEYS = ("iterations", "mg_only", "paper_schedule", "mg_only_ms_per_rhs", "paper_schedule_ms_per_rhs",
                   "speedup_vs_mg_only", "paper_schedule_speedup_vs_mg_only")


def _end_with_comparison(out: dict, mg_value: float, value: float, pp_value: float) -> dict:
    """Move the comparison the metric is about to the end of the JSON line, after every
    other workload: the headline's iterations, SL-MG alone and the paper's schedule, then
    their ms per RHS and the two speedups as scalars (COMPARISON_KEYS, in that order)."""
    for k in ("iterations", "mg_only", "paper_schedule"):
        out[k] = out.pop(k)
    out["mg_only_ms_per_rhs"] = out["mg_only"]["value"]
    out["paper_schedule_ms_per_rhs"] = out["paper_schedule"]["value"]
    out["speedup_vs_mg_only"] = round(mg_value / max(value, 1e-12), 3)
    out["paper_schedule_speedup_vs_mg_only"] = round(mg_value / max(pp_value, 1e-12), 3)
    return out


def run_gpu(args, rank: int, world: int):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_17486_gb300 as helm
    from paper_2306_17486_gb300 import _lib

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    kappas = _kappas(rank)
    probs, bs = [], []
    for k, kap in enumerate(kappas):
        oh = 2.0 * np.pi / (10.0 * float(kap.max()))   # 10 points per wavelength at max kappa
        probs.append(helm.Problem(torch.tensor(kap, dtype=torch.float32, device=dev), ABL, oh, levels=LEVELS))
        bs.append(torch.tensor(_rhs(rank, k), dtype=torch.complex64, device=dev))
    N = N_INT + 2 * ABL
    xs = [torch.zeros((N_RHS, N, N), dtype=torch.complex128, device=dev) for _ in range(N_MODELS)]
    net, train_info = _network(helm, dev, args)
    for p in probs:
        p.workspace(N_RHS, RESTART, net)

    def step(record=None, cnn=True, every=CNN_EVERY):
        for k in range(N_MODELS):
            xs[k].zero_()
            if cnn:
                net.set_problem(probs[k])      # encoder, once per slowness model (amortised)
            _, st = helm.fgmres_solve(probs[k], bs[k], xs[k], cnn=net if cnn else None, restart=RESTART,
                                      rtol=RTOL, maxit=MAXIT, warmup_iters=3, cnn_every=every)
            if record is not None:
                record.append(st)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # SL-MG-only arm (what the learned preconditioner is compared with)
    for _ in range(max(1, args.warmup // 2)):
        step(cnn=False)
    barrier()
    mg_stats = []
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m0.record()
    for _ in range(args.steps):
        step(mg_stats, cnn=False)
    m1.record()
    barrier()
    mg_ms = m0.elapsed_time(m1)
    mg_all = np.concatenate(mg_stats)
    # the paper's schedule (the network on every Arnoldi step)
    step(cnn=True, every=1)
    barrier()
    pp_stats = []
    m0.record()
    for _ in range(args.steps):
        step(pp_stats, cnn=True, every=1)
    m1.record()
    barrier()
    pp_ms = m0.elapsed_time(m1)
    pp_all = np.concatenate(pp_stats)
    for _ in range(args.warmup):
        step()
    barrier()
    L0 = _lib.lib().helm_launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    stats = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record()
    for _ in range(args.steps):
        step(stats)
    e1.record()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = int(_lib.lib().helm_launch_count() - L0)
    ms = max_over_ranks(ms, dist, dev)
    n_rhs_total = args.steps * N_MODELS * N_RHS * world
    value = ms / (args.steps * N_MODELS * N_RHS)   # per-rank wall time / per-rank RHS
    value_job = ms / (n_rhs_total)                  # whole-job ms per RHS
    allst = np.concatenate(stats)
    conv = float(np.mean(allst["status"] == 1))
    iters = allst["iters"]

    # ---- e2e: host buffers through the public API, copies inside the timed region ----
    hb = [b.cpu().pin_memory() for b in bs]
    hx = [torch.empty((N_RHS, N, N), dtype=torch.complex128).pin_memory() for _ in range(N_MODELS)]
    barrier()
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps // 2)):
        for k in range(N_MODELS):
            bd = hb[k].to(dev, non_blocking=True)
            xs[k].zero_()
            net.set_problem(probs[k])
            helm.fgmres_solve(probs[k], bd, xs[k], cnn=net, restart=RESTART, rtol=RTOL, maxit=MAXIT, warmup_iters=3,
                              cnn_every=CNN_EVERY)
            hx[k].copy_(xs[k], non_blocking=True)
    barrier()
    e2e_steps = max(1, args.steps // 2)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / (e2e_steps * N_MODELS * N_RHS)

    # ---- per-kernel shares of one profiled step (CUDA events around every launch) -------
    L = _lib.lib()
    import ctypes as C
    prof = _profile(L, C, step)
    tot_ms = sum(t[2] for t in prof)
    hbm, bf16, src = _peaks()
    # ---- rooflines: the step's dominant kernel and the other hot families, each timed
    #      live (library CUDA events on the launching stream) at the bench shape ----------
    roofs = _rooflines(helm, L, C, net, probs[0], dev, hbm, src, prof)
    dom = prof[0][0]
    roof = next((r for r in roofs if r["kernel"] == dom), roofs[0])

    mg_value = mg_ms / (args.steps * N_MODELS * N_RHS)
    pp_value = pp_ms / (args.steps * N_MODELS * N_RHS)
    out = {
        "metric": METRIC, "value": round(value_job, 4), "unit": "ms/RHS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 Hessenberg and solution)",
        "data": "synthetic: seeded GRF slowness (ell=8) in [0.25,1], seeded point sources",
        "config": {"workload": WORKLOAD, "grid": N, "interior": N_INT, "abl": ABL, "kappa_models": N_MODELS,
                   "rhs_per_model": N_RHS, "restart": RESTART, "rtol": RTOL, "mg_levels": LEVELS,
                   "preconditioner": "BF16 encoder-solver CNN (implicit layer) + FP32 SL-MG V(1,1) on every "
                                     f"{CNN_EVERY}rd Arnoldi step, SL-MG V(1,1) alone on the others, warm-up 3",
                   "cnn_every": CNN_EVERY,
                   "l2": "inputs larger than L2 (Krylov basis 1.9 GB/model)"},
        "method": "cnn+mg",
        "roofline": roof,
        "e2e": {"value": round(e2e_ms, 4), "unit": "ms/RHS",
                "h2d_bytes_per_step": int(sum(b.numel() * 8 for b in bs)),
                "d2h_bytes_per_step": int(sum(x.numel() * 16 for x in xs))},
        "gpu_launches": launches,
        "clocks": clk,
        "training": train_info,
    }
    if rank == 0:
        out["cpu_baseline"] = cpu_baseline(kappas[0], bs[0][:1].cpu().numpy(), float(iters.mean()))
    # compact per-kernel figures, then the comparison the metric is about, last
    out["roofline_kernels"] = [{k: r[k] for k in ("kernel", "bound", "achieved", "frac", "launch_ms", "share_of_step")}
                               for r in roofs if r is not roof]
    out["kernel_shares"] = [[n, c, round(t, 1), round(t / tot_ms, 3)] for n, c, t in prof[:6]]
    out["iterations"] = {"mean": round(float(iters.mean()), 1), "max": int(iters.max()), "converged_frac": conv,
                         "max_true_rel_res": float(allst["rel_res_true"].max())}
    out["mg_only"] = {"value": round(mg_value, 4), "unit": "ms/RHS",
                      "iterations_mean": round(float(mg_all["iters"].mean()), 1),
                      "iterations_max": int(mg_all["iters"].max()),
                      "converged_frac": float(np.mean(mg_all["status"] == 1))}
    out["paper_schedule"] = {"cnn_every": 1, "value": round(pp_value, 4), "unit": "ms/RHS",
                             "iterations_mean": round(float(pp_all["iters"].mean()), 1),
                             "iterations_max": int(pp_all["iters"].max()),
                             "converged_frac": float(np.mean(pp_all["status"] == 1)),
                             "max_true_rel_res": float(pp_all["rel_res_true"].max())}
    if not args.skip_1152:
        out["workload_1152"] = run_1152(helm, net, dev, rank)
    if not args.skip_serving:
        out["serving"] = run_serving()
    if not args.skip_ood:
        out["ood_shapes"] = run_ood(helm, net, dev, rank)
    if not args.skip_2176:
        out["workload_2176"] = run_2176(helm, net, dev, rank)
    _end_with_comparison(out, mg_value, value_job, pp_value)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


WEIGHTS = os.path.join(ROOT, "paper_2306_17486_gb300", "weights", "cnn_grf_multiscale.npz")

# Mixed-size serving: requests for 256^2, 512^2 and 1024^2 interiors (288^2, 576^2,
# 1152^2 nodes) interleaved, each its own layered+GRF model with 8 point sources,
# served by captured solver plans, one bucket per size on its own stream and thread
SERVE_SIZES, SERVE_REQUESTS, SERVE_BATCH = (256, 512, 1024), 3, 8


def run_serving():
    """p50 / p99 request latency and throughput of the serving path, with the network
    (on every CNN_EVERY-th step) and with SL-MG alone, on the same request stream."""
    from paper_2306_17486_gb300 import serving
    out = {"grids": [serving.bucket_config(n)[0] for n in SERVE_SIZES], "requests": SERVE_REQUESTS * len(SERVE_SIZES),
           "rhs_per_request": SERVE_BATCH, "arrival": "one burst, round robin over the sizes"}
    for key, mg_only in (("cnn_mg", False), ("mg_only", True)):
        rep = serving.run(SERVE_SIZES, SERVE_REQUESTS, SERVE_BATCH, mg_only=mg_only, cnn_every=CNN_EVERY)
        out[key] = {k: rep[k] for k in ("p50_ms", "p99_ms", "makespan_s", "throughput_rhs_per_s")}
        out[key]["iterations_mean"] = {g: v["iterations_mean"] for g, v in rep["per_grid"].items()}
        out[key]["converged_frac"] = min(v["converged_frac"] for v in rep["per_grid"].values())
        if rep["errors"]:
            out[key]["errors"] = rep["errors"][:3]
    return out


def _network(helm, dev, args):
    """The trained network: committed weights if present, else trained here (before any
    timing) with the same multiscale recipe."""
    from paper_2306_17486_gb300 import train as T
    import synth
    net = helm.Cnn(skip_threshold=256)
    path = args.weights or WEIGHTS
    if os.path.exists(path):
        meta = T.load_weights(net, path)
        return net, {"source": os.path.relpath(path, ROOT), "steps": meta.get("steps"),
                     "train_seconds": meta.get("seconds")}
    net.load_dict(synth.random_params(T.init_spec(net), seed=0))
    tr = T.Trainer(net, sizes=((128, 16, 3), (256, 32, 3), (576, 32, 4)), batch=32, steps=args.train_steps, seed=0,
                   pattern=(0, 2, 1, 2, 0, 2, 1, 2, 2, 2))
    t0 = time.time()
    tr.run(args.train_steps, log=None)
    torch.cuda.synchronize()
    return net, {"source": "trained in this run", "steps": args.train_steps, "train_seconds": time.time() - t0}


def _profile(L, C, fn):
    """Per-kernel (name, launches, total ms) of one call of fn under the library profiler."""
    import torch
    L.helm_profile_begin()
    fn()
    torch.cuda.synchronize()
    nk = C.c_int()
    L.helm_profile_end(C.byref(nk))
    prof = []
    for i in range(nk.value):
        nm, cnt, tot = C.c_char_p(), C.c_long(), C.c_double()
        L.helm_profile_read(i, C.byref(nm), C.byref(cnt), C.byref(tot))
        prof.append((nm.value.decode(), cnt.value, tot.value))
    prof.sort(key=lambda t: -t[2])
    return prof


def _rooflines(helm, L, C, net, P, dev, hbm, src, step_prof):
    """Achieved GB/s of the hot kernel families at the bench shape (64 RHS x 576^2):
    algorithmic bytes per launch (network layers, V-cycle levels, the matvec) over the
    average launch duration measured by the library's CUDA events on the launching stream,
    against the measured HBM copy bandwidth."""
    import torch
    N = P.nx
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    r = torch.randn((N_RHS, N, N), dtype=torch.complex64, device=dev, generator=g)
    net.set_problem(P)
    reps = 3
    for _ in range(2):
        net.apply(P, r)
        helm.slmg_vcycle(P, r)
        helm.helmholtz_apply(P, r)
    torch.cuda.synchronize()

    def run():
        for _ in range(reps):
            net.apply(P, r)
            helm.slmg_vcycle(P, r)
            helm.helmholtz_apply(P, r)

    prof = {n: (c, t) for n, c, t in _profile(L, C, run)}
    byts = dict(_net_layer_bytes(N, N_RHS))
    byts.update(_vcycle_bytes(N, LEVELS, N_RHS))
    byts["k_apply"] = 16.0 * N * N * N_RHS
    share = {n: t for n, _, t in step_prof}
    tot = sum(share.values())
    out = []
    for name, b in byts.items():
        if name not in prof:
            continue
        cnt, ms = prof[name]
        per_call = cnt / reps                      # launches per application
        t_launch = ms / cnt * 1e-3                 # average launch duration (s)
        b_launch = b / per_call                    # average algorithmic bytes per launch
        ach = b_launch / t_launch / 1e9
        tr = NCU_TRAFFIC_PER_RHS.get(name)
        out.append({"kernel": name, "bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(ach / hbm, 4), "peak_source": src, "bytes_per_launch": round(b_launch),
                    "launch_ms": round(t_launch * 1e3, 4),
                    "traffic": round(tr * N_RHS / per_call) if tr is not None else None,
                    "share_of_step": round(share.get(name, 0.0) / tot, 4) if tot else None})
    if "k_implicit" in prof:
        cnt, ms = prof["k_implicit"]
        t_launch = ms / cnt * 1e-3
        fl = _implicit_flops(N, N_RHS) / (cnt / reps)
        ach = fl / t_launch / 1e12
        out.append({"kernel": "k_implicit", "bound": "alu", "achieved": round(ach, 2), "peak": round(FP32_LANE_TFLOPS, 1),
                    "unit": "TFLOP/s", "frac": round(ach / FP32_LANE_TFLOPS, 4), "peak_source": "derived",
                    "flops_per_launch": round(fl), "launch_ms": round(t_launch * 1e3, 4), "traffic": None,
                    "share_of_step": round(share.get("k_implicit", 0.0) / tot, 4) if tot else None})
    out.sort(key=lambda d: -(d["share_of_step"] or 0.0))
    return out


ORACLE_ITERS = os.path.join(ROOT, "tests", "golden", "oracle_iterations_576.json")


def _oracle_network():
    """The committed trained weights in the oracle's own form (FP64 dicts): the flat
    parameter vector follows the parameter table order of the oracle's spec, BN running
    statistics are (mean, var) per BN in the same order."""
    from oracle import cnn as ocnn
    d = np.load(WEIGHTS)
    flat = d["params"].astype(np.float64)
    P, off = {}, 0
    for name, shape, *_ in ocnn.param_spec(16):
        n = int(np.prod(shape))
        P[name] = flat[off:off + n].reshape(shape)
        off += n
    assert off == flat.size, "weights file does not match the oracle's parameter table"
    run = d["running"].astype(np.float64)
    R, off = {}, 0
    for name, c in ocnn.bn_names(16):
        R[name] = (run[off:off + c], run[off + c:off + 2 * c])
        off += 2 * c
    return ocnn.Network(P, R, c0=16)


def _oracle_iteration_time(kappa, b1, cnn_its: int, mg_its: int):
    """Seconds per FGMRES(10) iteration of the FP64 oracle on one right-hand side: with
    the composed CNN + V-cycle preconditioner (cnn_its iterations) and with the V-cycle
    alone (mg_its iterations)."""
    from oracle import cnn as ocnn
    from oracle import fgmres as ofg
    from oracle import helmholtz as ohz
    from oracle import multigrid as omg
    from oracle import training as otr
    p = ohz.Problem(kappa, ABL)
    mg = omg.SLMultigrid(p, LEVELS)
    b = b1.astype(np.complex128)
    t_cnn = None
    if cnn_its > 0 and os.path.exists(WEIGHTS):
        net = _oracle_network()
        kf = ocnn.kappa_features(p.kappa, p.gamma)
        M = otr.composed_preconditioner(p, net, kf, mg)
        t0 = time.perf_counter()
        ofg.fgmres(p.A, b, np.zeros_like(b), M, RESTART, 0.0, cnn_its)
        t_cnn = (time.perf_counter() - t0) / cnn_its
    t0 = time.perf_counter()
    ofg.fgmres(p.A, b, np.zeros_like(b), mg, RESTART, 0.0, mg_its)
    t_mg = (time.perf_counter() - t0) / mg_its
    return t_cnn, t_mg


def _oracle_counts():
    try:
        with open(ORACLE_ITERS) as f:
            d = json.load(f)
        return d.get("mean_iterations"), d.get("cnn_mg", {}).get("mean_iterations")
    except OSError:
        return None, None


def cpu_baseline(kappa, b1, gpu_iters_mean):
    """The FP64 oracle as it stands, on this host, for a bounded sample of the workload:
    FGMRES(10) iterations on one right-hand side of kappa 0 with the composed
    preconditioner (the trained network through the oracle's forward, then the
    V-cycle), scaled to ms per RHS by the GPU run's mean iteration count."""
    t_cnn, t_mg = _oracle_iteration_time(kappa, b1[0], 2, 6)
    threads = int(os.environ.get("OMP_NUM_THREADS", "0") or 0) or (os.cpu_count() or 1)
    # the headline schedule: the network on Arnoldi steps j = 0 mod CNN_EVERY of each cycle
    f_cnn = len(range(0, RESTART, CNN_EVERY)) / RESTART
    per_it = f_cnn * t_cnn + (1 - f_cnn) * t_mg if t_cnn is not None else t_mg
    return {"value": round(per_it * gpu_iters_mean * 1e3, 2), "unit": "ms/RHS", "cores": threads,
            "kind": "oracle",
            "sample": f"2 CNN+V-cycle FGMRES(10) iterations ({t_cnn:.2f} s each) and 6 V-cycle-only iterations "
                      f"({t_mg:.3f} s each) on 1 RHS of kappa 0, mixed {f_cnn:.1f} : {1 - f_cnn:.1f} as in the "
                      f"schedule, x mean GPU iterations/RHS {gpu_iters_mean:.1f}"
            if t_cnn is not None else f"6 V-cycle FGMRES(10) iterations on 1 RHS ({t_mg:.3f} s each)"}


def run_reference(args, rank: int, world: int):
    """Reference arm: the FP64 oracle on the host cores (there is no upstream code), on
    this workload's first right-hand side: each step runs one FGMRES(10) iteration with
    the composed CNN + V-cycle preconditioner; ms per RHS = the per-iteration time x the
    oracle's own iteration count to 1e-6 (stored by tests/golden/make_oracle_iterations.py,
    which calls only the oracle)."""
    if rank != 0:
        return
    from oracle import cnn as ocnn
    from oracle import fgmres as ofg
    from oracle import helmholtz as ohz
    from oracle import multigrid as omg
    from oracle import training as otr
    kap = _kappas(0)[0]
    b = _rhs(0, 0)[0].astype(np.complex128)
    p = ohz.Problem(kap, ABL)
    mg = omg.SLMultigrid(p, LEVELS)
    net = _oracle_network()
    kf = ocnn.kappa_features(p.kappa, p.gamma)
    M = otr.composed_preconditioner(p, net, kf, mg)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        ofg.fgmres(p.A, b, np.zeros_like(b), M, RESTART, 0.0, 1)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    per_it = float(np.mean(times))
    n_mg, n_cnn = _oracle_counts()
    n_it = n_cnn if n_cnn else n_mg
    which = "CNN+V-cycle" if n_cnn else "V-cycle-only (CNN+V-cycle count not stored)"
    v = per_it * n_it * 1e3
    threads = int(os.environ.get("OMP_NUM_THREADS", "0") or 0) or (os.cpu_count() or 1)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 2), "unit": "ms/RHS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per_it * 1e3, 1),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: seeded GRF slowness (ell=8) in [0.25,1], seeded point sources",
        "config": {"workload": WORKLOAD, "grid": N_INT + 2 * ABL, "interior": N_INT, "abl": ABL,
                   "restart": RESTART, "rtol": RTOL, "mg_levels": LEVELS},
        "cpu_baseline": {"value": round(v, 2), "unit": "ms/RHS", "cores": threads, "kind": "oracle",
                         "sample": f"1 CNN+V-cycle FGMRES(10) iteration of the FP64 oracle per step on RHS 0 of "
                                   f"kappa 0 (the paper's schedule: the network on every step), x {n_it:.1f} "
                                   f"iterations ({which} count of the oracle to 1e-6)"},
        "e2e": {"value": round(v, 2), "unit": "ms/RHS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native")
    ap.add_argument("--weights", default=None)
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--skip-1152", action="store_true", help="leave out the 1152^2 (1024^2 interior) workload")
    ap.add_argument("--skip-serving", action="store_true", help="leave out the mixed-size serving run")
    ap.add_argument("--skip-2176", action="store_true", help="leave out the 2176^2 (2048^2 interior) workload")
    ap.add_argument("--skip-ood", action="store_true",
                    help="leave out the rectangular out-of-distribution shapes (512 x 1024, 352 x 800)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
