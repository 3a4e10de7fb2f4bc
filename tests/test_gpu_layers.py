"""Element-by-element GPU parity of single network layers through their C-ABI entry
points, against the FP64 oracle on the GPU's rounded inputs, plus the whole network
at the benchmark's shape.

* The fused inverted bottleneck (Section 4.4, MobileNetV2 block; helm_ib_bf16) at
  C = 16, 32, 64 on grids with ragged tiles (the kernel tiles 8 x 16 outputs).
* The implicit layer (Section 4.2, Eq. 14; helm_implicit_bf16) at m = 8, 36 and 72.
* The network forward at I = 576 with the layer plan the benchmark runs (coarsest
  level I/16, batch 8, the persistent kernels wrapping over their segments).

Per-element bounds follow the kernels' arithmetic (u16 = 2^-11 for FP16, ub = 2^-8
for the BF16 rounding of a stored activation, doubled for margin):
* bottleneck: the FP16 expanded activations and FP16 row sums of the depthwise stage
  perturb its output by at most 3 u16 sum |w_dw||h| (h the expanded activation);
  the depthwise output is stored in BF16 (ub |a|), so each projection input a_k is off
  by at most ub (|a_k| + |s1_k| D_k), D_k = sum |w_dw||h|; the projection sums these
  with |w_p|, BN2 scales by |s2|, and the output is rounded to BF16:
      |y - y_ref| <= ub |y_ref| + ub |s2| sum_k |w_p| (|a_k| + |s1_k| D_k);
* implicit layer: four dense DFT stages of length 2m in FP32, each adding at most
  2m eps32 of the magnitude bound max|G_hat| sum|x|, then BF16 rounding:
      |y - y_ref| <= ub |y_ref| + 4 (2m) 2^-24 max|G_hat| sum|x|.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import cnn as ocnn
from oracle import helmholtz as ohz
from oracle import implicit as oimp

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
UB = 2.0 ** -8


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_17486_gb300 as h
    return h


def _bf(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32).to(torch.bfloat16).double().numpy()


def _f16(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32).to(torch.float16).double().numpy()


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("C,B,H,W", [(16, 2, 17, 23), (16, 1, 144, 144), (32, 2, 37, 29), (32, 3, 72, 72),
                                     (64, 2, 18, 18), (64, 4, 36, 36), (64, 1, 9, 40)])
def test_fused_inverted_bottleneck_matches_oracle_per_element(helm, C, B, H, W):
    rng = np.random.default_rng(C * 1000 + H)
    E = 6 * C
    x = _bf(rng.standard_normal((B, C, H, W)))
    w_exp = _bf(rng.standard_normal((E, C)) / np.sqrt(C))
    w_dw = _f16(rng.standard_normal((E, 3, 3)) / 3.0)          # the kernel keeps them in FP16
    w_proj = _bf(rng.standard_normal((C, E)) / np.sqrt(E))
    P = {"ib.exp.w": w_exp, "ib.dw.w": w_dw, "ib.proj.w": w_proj}
    running, fold = {}, {}
    for nm, c in (("ib.bn0", E), ("ib.bn1", E), ("ib.bn2", C)):
        sc, sh = _f32(rng.uniform(0.5, 1.5, c)), _f32(0.3 * rng.standard_normal(c))
        # running statistics (0, 1 - eps) make the oracle's fold exactly (sc, sh)
        P[nm + ".g"], P[nm + ".b"] = sc, sh
        running[nm] = (np.zeros(c), np.full(c, 1.0 - ocnn.BN_EPS))
        fold[nm] = np.concatenate([sc, sh]).astype(np.float32)
    tp = ocnn.Tape(P, record=False)
    xv = ocnn.Var(x)
    h = ocnn.softplus(tp, ocnn.batchnorm(tp, ocnn.conv1x1(tp, xv, "ib.exp.w"), "ib.bn0", False, running))
    d = ocnn.depthwise3x3(tp, h, "ib.dw.w")
    a = ocnn.softplus(tp, ocnn.batchnorm(tp, d, "ib.bn1", False, running))
    z = ocnn.batchnorm(tp, ocnn.conv1x1(tp, a, "ib.proj.w"), "ib.bn2", False, running)
    y_ref = x + z.a
    # the same block through the oracle's own composition (checks the staging above)
    y_ib = ocnn.inverted_bottleneck(ocnn.Tape(P, record=False), ocnn.Var(x), "ib", False, running).a
    assert np.array_equal(y_ib, y_ref)
    # magnitude terms of the bound
    Dk = ocnn.depthwise3x3(ocnn.Tape({"w": np.abs(w_dw)}, record=False), ocnn.Var(np.abs(h.a)), "w").a
    s1 = np.abs(P["ib.bn1.g"])[None, :, None, None]
    s2 = np.abs(P["ib.bn2.g"])[None, :, None, None]
    prop = np.einsum("ok,bkhw->bohw", np.abs(w_proj), np.abs(a.a) + s1 * Dk)
    bound = UB * np.abs(y_ref) + UB * s2 * prop

    dev = "cuda"
    T = lambda v, dt=torch.float32: torch.tensor(np.ascontiguousarray(v), dtype=dt, device=dev)
    xg = T(np.transpose(x, (0, 2, 3, 1))).to(torch.bfloat16).contiguous()
    yg = torch.empty_like(xg)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
    L = helm.lib()
    helm._lib.check(L.helm_ib_bf16(helm._ptr(xg), B, H, W, C, helm._ptr(T(w_exp)), helm._ptr(T(fold["ib.bn0"])),
                                   helm._ptr(T(w_dw)), helm._ptr(T(fold["ib.bn1"])), helm._ptr(T(w_proj)),
                                   helm._ptr(T(fold["ib.bn2"])), helm._ptr(yg), helm._ptr(ws), ws.numel(),
                                   helm._stream()), "helm_ib_bf16")
    y = np.transpose(yg.double().cpu().numpy(), (0, 3, 1, 2))
    err = np.abs(y - y_ref)
    worst = float((err / bound).max())
    assert worst <= 1.0, (worst, float(err.max()), float(np.abs(y_ref).max()))
    assert helm.device_errors() == 0


@pytest.mark.parametrize("m,B", [(8, 3), (36, 2), (72, 1)])
def test_implicit_layer_matches_oracle_per_element(helm, m, B):
    C = 64
    nk = C // 2
    rng = np.random.default_rng(m)
    K = np.stack([np.broadcast_to(oimp.laplacian_plus_i().real, (nk, 3, 3)),
                  np.broadcast_to(oimp.laplacian_plus_i().imag, (nk, 3, 3))]).copy()
    K += 0.2 * rng.standard_normal(K.shape)
    ghat = np.stack([oimp.greens_hat(K[0, k] + 1j * K[1, k], m) for k in range(nk)])
    ghat = ghat.astype(np.complex64).astype(np.complex128)            # the GPU reads complex64
    x = _bf(rng.standard_normal((B, C, m, m)))
    tp = ocnn.Tape({}, record=False)
    y_ref = ocnn.implicit_layer(tp, ocnn.Var(x), "unused", ghat).a
    xs = x[:, :nk] + 1j * x[:, nk:]
    mag = np.abs(xs).sum(axis=(2, 3))                                   # [B, nk]
    gmax = np.abs(ghat).max(axis=(1, 2))                                # [nk]
    tail = 4 * (2 * m) * 2.0 ** -24 * gmax[None, :] * mag               # [B, nk]
    tail = np.concatenate([tail, tail], axis=1)[:, :, None, None]
    bound = UB * np.abs(y_ref) + tail

    xg = torch.tensor(np.transpose(x, (0, 2, 3, 1)), dtype=torch.float32, device="cuda").to(torch.bfloat16)
    xg = xg.contiguous()
    yg = torch.empty_like(xg)
    gg = torch.tensor(ghat, dtype=torch.complex64, device="cuda")
    helm._lib.check(helm.lib().helm_implicit_bf16(helm._ptr(xg), B, m, C, helm._ptr(gg), helm._ptr(yg),
                                                  helm._stream()), "helm_implicit_bf16")
    y = np.transpose(yg.double().cpu().numpy(), (0, 3, 1, 2))
    worst = float((np.abs(y - y_ref) / bound).max())
    assert worst <= 1.0, worst


def test_network_forward_at_the_benchmark_shape(helm):
    """I = 576 (512^2 plus the 32-cell layer), skip threshold 256 (coarsest level I/16 =
    36, the benchmark's plan), batch 8, the committed trained weights: the GPU network
    against the oracle's forward on samples 0 and 7 (the eval-mode forward treats
    samples independently).  The GPU rounds some 40 stored activations to BF16; the
    2-norm error is bounded by 2 % (about sqrt(40) BF16 roundings of relative 2^-9
    with a gain of 2), every element by 2^-4 |ref| + 2^-4 RMS(ref)."""
    from paper_2306_17486_gb300 import train as T
    net = helm.Cnn(skip_threshold=256)
    T.load_weights(net, os.path.join(ROOT, "paper_2306_17486_gb300", "weights", "cnn_grf_multiscale.npz"))
    d = np.load(os.path.join(ROOT, "paper_2306_17486_gb300", "weights", "cnn_grf_multiscale.npz"))
    I, abl, B = 576, 32, 8
    kap = synth.grf_kappa(512, abl, 8.0, seed=10).astype(np.float32).astype(np.float64)
    oh = 2 * np.pi / 10 / kap.max()
    p = helm.Problem(torch.tensor(kap, dtype=torch.float32, device="cuda"), abl, oh, levels=4)
    net.set_problem(p)
    r = synth.random_complex((B, I, I), 12).astype(np.complex64).astype(np.complex128)
    e = net.apply(p, torch.tensor(r, dtype=torch.complex64, device="cuda")).cpu().numpy()
    # the oracle with the GPU's BF16 conv weights
    flat = d["params"].astype(np.float64)
    Pd, off = {}, 0
    for name, shape, *_ in ocnn.param_spec(16):
        n = int(np.prod(shape))
        v = flat[off:off + n].reshape(shape)
        Pd[name] = _bf(v) if (name.endswith(".w") and v.ndim in (2, 4) and name != "s.proj.w") else v
        off += n
    run = d["running"].astype(np.float64)
    R, off = {}, 0
    for name, c in ocnn.bn_names(16):
        R[name] = (run[off:off + c], run[off + c:off + 2 * c])
        off += 2 * c
    on = ocnn.Network(Pd, R, c0=16)
    op = ohz.Problem(kap, abl, omega_h=oh)
    kf = ocnn.kappa_features(op.kappa, op.gamma.astype(np.float32).astype(np.float64))
    for i in (0, B - 1):
        ref, _ = on.forward(r[i:i + 1], kf, train=False, skip=False)
        ref = ref[0]
        err = np.linalg.norm(e[i] - ref) / np.linalg.norm(ref)
        assert err < 2e-2, (i, err)
        rms = np.sqrt(np.mean(np.abs(ref) ** 2))
        worst = float((np.abs(e[i] - ref) / (2.0 ** -4 * (np.abs(ref) + rms))).max())
        assert worst <= 1.0, (i, worst, err)
