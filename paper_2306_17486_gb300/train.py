"""Multiscale training of the encoder-solver network on residual/error pairs generated
by the plain SL-multigrid FGMRES (Section 4.3, Eq. 16-17; Section 5.3).

Pairs are normalised by the residual's RMS over the grid (the library's reading of the
unstated input scale), so inputs are O(1) at every grid size.

Every step: `kappas_per_batch` slowness models from a seeded pool of the step's grid size
(absorbing layer included, gamma = 0.05 as in Section 4.3; Eq. 16: each pair carries
its own kappa, so BatchNorm statistics average over models), a batch of random smooth-plus-noise
vectors x (inputs: drawn with a seeded torch generator on the device), per-sample
iteration counts k ~ U{2..20}, then on the library's kernels:
    (e, r) = Eq. (17) pairs, normalised by RMS(r)     helm_datagen_pairs
    e_pred = Net(r) with batch-statistics BN          helm_cnn_apply(train=1)
    loss, dL/de = Eq. (16)                            helm_mse_loss
    dL/dtheta                                         helm_cnn_precond_backward
    Adam                                              helm_adam_step
The multiscale schedule alternates the grid size in blocks of steps (Section 4.3:
datasets switched every few epochs, larger sizes shorter), six small blocks for every
four large ones.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np
import torch

from . import Adam, Cnn, Problem, datagen_pairs, mse_loss, training_field


def smooth_plus_noise(B: int, N: int, gen: torch.Generator, ell: float = 4.0, noise: float = 0.1,
                      device="cuda") -> torch.Tensor:
    """Random training vectors: complex Gaussian random field (Gaussian filter of std
    ell/sqrt(2), periodic) scaled to unit RMS, plus `noise` x complex white noise.  The
    standard normal numbers are drawn here; the filter, scaling and sum run in the
    library (helm_training_field)."""
    white = torch.randn((B, 4, N, N), generator=gen, device=device)
    return training_field(white, ell / math.sqrt(2.0), noise)


class Trainer:
    """sizes: ((N_total, abl[, levels]), ...) grids including the absorbing layer, with
    the V-cycle depth of the data generation (default `levels`); pattern: the size index
    of each block of `block` steps, repeated (default: six small blocks for every four
    large ones with two sizes, round robin otherwise)."""

    def __init__(self, net: Cnn, sizes=((128, 16), (256, 16)), batch: int = 32, lr: float = 1e-3,
                 steps: int = 2000, seed: int = 0, pool: int = 24, levels: int = 3, kappa_ell: float = 8.0,
                 block: int = 100, kappas_per_batch: int = 4, pattern=None, device="cuda"):
        import synth
        self.net, self.batch, self.steps, self.block = net, batch, steps, block
        self.G = kappas_per_batch
        self.lr0 = lr
        self.device = torch.device(device)
        self.gen = torch.Generator(device=self.device)
        self.gen.manual_seed(seed)
        self.rng = np.random.default_rng(seed)
        self.pools = []
        if pattern is not None:
            self.PATTERN = tuple(pattern)
        elif len(sizes) > 2:
            self.PATTERN = tuple(range(len(sizes)))
        for si, size in enumerate(sizes):
            N, abl = size[0], size[1]
            lv = size[2] if len(size) > 2 else levels
            probs = []
            for j in range(pool):
                kap = synth.grf_kappa(N - 2 * abl, abl, kappa_ell, seed=100000 * (si + 1) + j + 1000 * seed)
                oh = 2 * np.pi / (10.0 * float(kap.max()))
                probs.append(Problem(torch.tensor(kap, dtype=torch.float32, device=self.device), abl, oh,
                                     gamma0=0.05, levels=lv))
            self.pools.append(probs)
        self.opt = Adam(net.params, lr=lr)
        self.step_i = 0
        self.history = []

    # six blocks of the small size for every four of the large one (16000 : 10000)
    PATTERN = (0, 1, 0, 1, 0, 1, 0, 1, 0, 0)

    def size_index(self, step: int) -> int:
        if len(self.pools) == 1:
            return 0
        return self.PATTERN[(step // self.block) % len(self.PATTERN)] % len(self.pools)

    def lr_at(self, step: int) -> float:
        # lr 1e-3, divided by 10 at 75% of the run (Section 5.3: /10 every 100 of 250 epochs)
        return self.lr0 if step < int(0.75 * self.steps) else self.lr0 / 10

    def step(self) -> float:
        i = self.step_i
        si = self.size_index(i)
        pool = self.pools[si]
        probs = [pool[int(j)] for j in self.rng.choice(len(pool), size=self.G, replace=False)]
        N = probs[0].nx
        per = self.batch // self.G
        es, rs = [], []
        for p in probs:   # Eq. (17) pairs, `per` samples for each slowness model
            x = smooth_plus_noise(per, N, self.gen, device=self.device)
            k = torch.randint(2, 21, (per,), generator=self.gen, device=self.device, dtype=torch.int32)
            e1, r1 = datagen_pairs(p, x, k, max_iters=20, normalise=True)
            es.append(e1)
            rs.append(r1)
        e, r = torch.cat(es), torch.cat(rs)
        e_pred = self.net.forward_train(probs, r)
        loss, g = mse_loss(e_pred, e)
        grads = self.net.backward(probs, g)
        self.opt.lr = self.lr_at(i)
        self.opt.step(grads)
        self.net.set_params()
        self.step_i += 1
        return loss

    def run(self, steps: int | None = None, log_every: int = 100, log=print):
        steps = self.steps if steps is None else steps
        t0 = time.time()
        losses = []
        for _ in range(steps):
            losses.append(self.step())
            if self.step_i % log_every == 0:
                lv = float(torch.stack(losses[-log_every:]).mean().item())
                self.history.append((self.step_i, self.size_index(self.step_i - 1), lv))
                if log:
                    log(f"step {self.step_i:6d} size {self.pools[self.size_index(self.step_i - 1)][0].nx:4d} "
                        f"loss {lv:.5f} lr {self.lr_at(self.step_i - 1):.0e} {time.time() - t0:7.1f}s")
        return self.history

    # ---- checkpoint ------------------------------------------------------------------
    def save(self, path: str):
        np.savez(path, params=self.net.params.cpu().numpy(), running=self.net.running_dict_flat(),
                 adam_m=self.opt.m.cpu().numpy(), adam_v=self.opt.v.cpu().numpy(), adam_t=self.opt.t,
                 step=self.step_i, gen_state=self.gen.get_state().cpu().numpy(),
                 rng_state=np.frombuffer(json.dumps(self.rng.bit_generator.state).encode(), dtype=np.uint8),
                 history=np.array(self.history, dtype=np.float64).reshape(-1, 3))

    def load(self, path: str):
        d = np.load(path)
        self.net.params.copy_(torch.from_numpy(d["params"]))
        self.net.set_params()
        self.net.load_running_flat(d["running"])
        self.opt.m.copy_(torch.from_numpy(d["adam_m"]))
        self.opt.v.copy_(torch.from_numpy(d["adam_v"]))
        self.opt.t = int(d["adam_t"])
        self.step_i = int(d["step"])
        self.gen.set_state(torch.from_numpy(d["gen_state"]))
        self.rng.bit_generator.state = json.loads(bytes(d["rng_state"]).decode())
        self.history = [tuple(h) for h in d["history"]]


def retrain(net: Cnn, problem: Problem, steps: int = 300, batch: int = 32, lr: float = 1e-4, seed: int = 0,
            log=None) -> list:
    """Solve-time re-training on one (out-of-distribution) slowness model (Section 5:
    the pre-trained network is optimised for a short time on the problem at hand):
    Adam on Eq. (17) pairs generated from `problem` by the plain solver, batches of
    `batch` samples of that single model, constant learning rate.  `problem` must be
    built with gamma0 = 0.05 as in the training data (Section 4.3).  Returns the losses."""
    gen = torch.Generator(device=problem.device)
    gen.manual_seed(seed)
    opt = Adam(net.params, lr=lr)
    N = problem.nx
    losses = []
    for i in range(steps):
        x = smooth_plus_noise(batch, N, gen, device=problem.device)
        k = torch.randint(2, 21, (batch,), generator=gen, device=problem.device, dtype=torch.int32)
        e, r = datagen_pairs(problem, x, k, max_iters=20, normalise=True)
        e_pred = net.forward_train([problem], r)
        loss, g = mse_loss(e_pred, e)
        grads = net.backward([problem], g)
        opt.step(grads)
        net.set_params()
        losses.append(loss)
        if log and (i + 1) % 50 == 0:
            log(f"retrain step {i + 1}: loss {float(torch.stack(losses[-50:]).mean()):.4f}")
    return [float(v) for v in losses]


def save_weights(net: Cnn, path: str, meta: dict | None = None):
    """Trained network for inference: FP32 parameters and BN running statistics."""
    np.savez(path, params=net.params.cpu().numpy(), running=net.running_dict_flat(),
             meta=np.frombuffer(json.dumps(meta or {}).encode(), dtype=np.uint8))


def load_weights(net: Cnn, path: str) -> dict:
    d = np.load(path)
    net.params.copy_(torch.from_numpy(d["params"]))
    net.set_params()
    net.load_running_flat(d["running"])
    return json.loads(bytes(d["meta"]).decode()) if "meta" in d else {}


def init_spec(net: Cnn):
    """(name, shape, fan_in, kind[, values]) for every parameter, from the library's own
    table: PyTorch's default Kaiming-uniform initialisation of convolutions (fan_in =
    dim1 x kernel area, also for transposed convolutions), BN gamma = 1 and beta = 0,
    and the implicit kernels set to L + iI (Section 5.3)."""
    L = np.array([[0, -1, 0], [-1, 4, -1], [0, -1, 0]], dtype=np.float64)
    spec = []
    for name, shape, _ in net.spec:
        if name.endswith(".g"):
            spec.append((name, shape, 0, "bn_g"))
        elif name.endswith(".b") and not name.startswith("s.proj"):
            spec.append((name, shape, 0, "bn_b"))
        elif name == "s.imp.K":
            nk = shape[1]
            re = np.broadcast_to(L, (nk, 3, 3))
            im = np.broadcast_to(np.eye(3)[1:2, :].T @ np.eye(3)[1:2, :], (nk, 3, 3))  # delta at the centre
            spec.append((name, shape, 0, "fixed", np.stack([re, im]).ravel()))
        elif name == "s.proj.b":
            spec.append((name, shape, 16, "bias"))
        else:
            area = 9 if len(shape) == 4 else (9 if len(shape) == 3 else 1)
            fan_in = (shape[1] if len(shape) != 3 else 1) * area
            spec.append((name, shape, fan_in, "w"))
    return spec


def main():
    import argparse
    import os
    import sys
    ap = argparse.ArgumentParser(description="multiscale training of the encoder-solver network")
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--sizes", default="128:16,256:32",
                    help="N_total:absorbing-layer cells[:V-cycle levels], comma separated")
    ap.add_argument("--pattern", default=None, help="size index per block of 100 steps, comma separated")
    ap.add_argument("--skip-threshold", type=int, default=256)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--init", default=None, help="start from these weights (fine-tuning)")
    ap.add_argument("--explicit", action="store_true", help="the explicit U-Net (no implicit step, Section 6)")
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synth
    net = Cnn(skip_threshold=a.skip_threshold, explicit_unet=a.explicit)
    prev = {}
    if a.init:
        prev = load_weights(net, a.init)
    else:
        net.load_dict(synth.random_params(init_spec(net), seed=a.seed))
    sizes = tuple(tuple(int(v) for v in t.split(":")) for t in a.sizes.split(","))
    pattern = tuple(int(v) for v in a.pattern.split(",")) if a.pattern else None
    tr = Trainer(net, sizes=sizes, batch=a.batch, steps=a.steps, seed=a.seed, lr=a.lr, pattern=pattern)
    t0 = time.time()
    hist = tr.run(a.steps)
    torch.cuda.synchronize()
    dt = time.time() - t0
    meta = {"steps": a.steps + int(prev.get("steps") or 0), "batch": a.batch, "sizes": a.sizes,
            "pattern": a.pattern, "seed": a.seed, "lr": a.lr, "skip_threshold": a.skip_threshold,
            "explicit_unet": bool(a.explicit),
            "seconds": dt + float(prev.get("seconds") or 0.0), "history": [list(h) for h in hist]}
    if a.init:
        meta["init"] = {k: prev.get(k) for k in ("steps", "sizes", "seconds")}
    save_weights(net, a.out, meta)
    print(f"trained {a.steps} steps in {dt:.1f} s -> {a.out}")


if __name__ == "__main__":
    main()
