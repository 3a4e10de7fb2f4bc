"""Pins of the oracle's encoder-solver network (Sections 4.1-4.4, 5.3): gradients
against central finite differences, shapes and parameter counts printed in the
paper, BatchNorm folding, and the data-generation / loss / Adam steps (no GPU)."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import cnn
from oracle import helmholtz as hz
from oracle import multigrid as mg
from oracle import training as tr

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _setup(I=32, B=2, c0=4, seed=1, implicit=True):
    P = synth.random_params(cnn.param_spec(c0, implicit=implicit), seed=seed, bn_jitter=0.2)
    net = cnn.Network(P, c0=c0, implicit=implicit)
    abl = 4
    prob = hz.Problem(synth.grf_kappa(I - 2 * abl, abl, 4.0, seed + 1), abl)
    kf = cnn.kappa_features(prob.kappa, prob.gamma)
    r = synth.random_complex((B, I, I), seed + 2)
    et = 0.01 * synth.random_complex((B, I, I), seed + 3)
    return net, P, kf, r, et


@pytest.mark.parametrize("implicit", [True, False], ids=["implicit", "explicit"])
@pytest.mark.parametrize("skip", [True, False])
def test_network_gradients_match_central_differences(skip, implicit):
    """Every parameter tensor: directional derivative of the Eq. (16) loss along a
    random direction, analytic vs central differences (FP64), relative 1e-6; for the
    implicit U-Net and for the explicit U-Net of Section 6."""
    net, P, kf, r, et = _setup(implicit=implicit)

    def loss_of(params):
        net.params = params
        e, _ = net.forward(r, kf, train=True, skip=skip)
        return tr.mse_loss(e, et)[0]

    net.params = P
    e, tp = net.forward(r, kf, train=True, skip=skip, record=True)
    L, ge = tr.mse_loss(e, et)
    grads = net.backward(tp, ge)
    rng = np.random.default_rng(0)
    assert set(grads) == set(P)
    for name in P:
        d = rng.standard_normal(P[name].shape)
        # 4-point central difference (truncation O(h^4))
        vals = []
        for c in (2, 1, -1, -2):
            Q = dict(P)
            Q[name] = P[name] + c * 1e-4 * d
            vals.append(loss_of(Q))
        fd = (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * 1e-4)
        an = float((grads[name] * d).sum())
        assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-10 * abs(L)), (name, fd, an)


def test_parameter_count_and_feature_shapes_match_paper():
    n_solver = sum(int(np.prod(s)) for n, s, *_ in cnn.param_spec(16) if n.startswith("s."))
    ref = GOLD["solver_params"]["value"]
    assert abs(n_solver - ref) / ref < 0.03          # 360K (Table 4)
    n_expl = sum(int(np.prod(s)) for n, s, *_ in cnn.param_spec(16, implicit=False) if n.startswith("s."))
    ref_e = GOLD["explicit_solver_params"]["value"]
    assert abs(n_expl - ref_e) / ref_e < 0.03        # 360K (Table 4, explicit model)
    # the two differ by the 32 complex 3x3 kernels of the implicit step (Section 4.2)
    assert n_solver - n_expl == 32 * 9 * 2
    P = synth.random_params(cnn.param_spec(16), seed=0)
    net = cnn.Network(P, c0=16)
    I = 64
    tp = cnn.Tape(P, record=False)
    kf = cnn.Var(np.zeros((1, 2, I, I)))
    encs = cnn.encoder(tp, kf, False, net.running)
    for (c, div), enc in zip(GOLD["encoder_feature_maps"]["value"], encs):
        assert enc.a.shape == (1, c, I // div, I // div)
    assert cnn.coarsest_size(1024) == 1024 // GOLD["solver_coarsest"]["value"][1]
    assert cnn.coarsest_size(256) == 256 // 8
    assert cnn.skip_last_down(GOLD["skip_threshold"]["value"] - 1)
    assert not cnn.skip_last_down(GOLD["skip_threshold"]["value"])


def test_explicit_unet_is_the_implicit_one_with_an_identity_step():
    """Section 6's explicit U-Net is the implicit network without the implicit step.
    With G_hat = 1 the implicit step crop(IFFT(FFT(pad(x)))) is the identity, so the
    two networks must agree on the same parameters: outputs in training and in
    evaluation mode, and every shared parameter's gradient."""
    net_i, P, kf, r, et = _setup(implicit=True)
    nk = P["s.imp.K"].shape[1]
    net_i.ghat = lambda m: np.ones((nk, 2 * m, 2 * m), dtype=np.complex128)
    Pe = {k: v for k, v in P.items() if k != "s.imp.K"}
    net_e = cnn.Network(Pe, c0=4, implicit=False)
    assert set(P) - set(Pe) == {"s.imp.K"}
    assert [n for n, *_ in cnn.param_spec(4, implicit=False)] == [n for n, *_ in cnn.param_spec(4) if n != "s.imp.K"]
    for skip in (True, False):
        ei, _ = net_i.forward(r, kf, train=False, skip=skip)
        ee, _ = net_e.forward(r, kf, train=False, skip=skip)
        assert np.abs(ee - ei).max() <= 1e-12 * np.abs(ei).max()
        ei, ti = net_i.forward(r, kf, train=True, skip=skip, record=True)
        ee, te = net_e.forward(r, kf, train=True, skip=skip, record=True)
        assert np.abs(ee - ei).max() <= 1e-12 * np.abs(ei).max()
        gi = net_i.backward(ti, tr.mse_loss(ei, et)[1])
        ge = net_e.backward(te, tr.mse_loss(ee, et)[1])
        assert set(ge) == set(Pe)
        for k in Pe:
            assert np.abs(ge[k] - gi[k]).max() <= 1e-10 * max(np.abs(gi[k]).max(), 1e-300), k
    # the implicit step is not the identity for the real G_hat (L + iI kernels)
    net_r = cnn.Network(P, c0=4)
    assert np.abs(net_r.forward(r, kf)[0] - net_e.forward(r, kf)[0]).max() > 1e-3 * np.abs(ei).max()


def test_implicit_step_reaches_the_whole_map_and_the_explicit_network_does_not():
    """Section 4.2: the implicit step widens the field of view.  A change of the solver
    input at one corner of the I/2 map (I = 256) is followed to the opposite corner of
    the output.
    * The explicit U-Net's receptive field (3x3 convolutions at strides 1-8 and back,
      about 105 pixels of the 128-pixel map) does not reach it: bitwise unchanged.
    * Through the implicit layer the reach is set by the learned kernel.  With K = L +
      1e-3 i delta (a weakly shifted Laplacian, Green's function decaying over about 30
      coarse pixels) the change is orders of magnitude above that of the initial
      L + iI (a kernel about a pixel wide, the change at rounding level).  Both go
      through the same up path, whose random weights attenuate either equally."""
    I, c0 = 256, 4
    P = synth.random_params(cnn.param_spec(c0), seed=3, bn_jitter=0.2)
    nk = P["s.imp.K"].shape[1]
    lap = np.array([[0.0, -1.0, 0.0], [-1.0, 4.0, -1.0], [0.0, -1.0, 0.0]])
    weak = np.zeros((3, 3))
    weak[1, 1] = 1e-3
    P_long = dict(P)
    P_long["s.imp.K"] = np.stack([np.broadcast_to(lap, (nk, 3, 3)), np.broadcast_to(weak, (nk, 3, 3))]).copy()
    Pe = {k: v for k, v in P.items() if k != "s.imp.K"}
    rng = np.random.default_rng(4)
    kf = rng.uniform(0.0625, 1.0, size=(1, 2, I, I))
    x0 = rng.standard_normal((1, 2, I // 2, I // 2))
    x1 = x0.copy()
    x1[0, :, 0, 0] += 1.0

    def far_change(params, implicit):
        net = cnn.Network(params, c0=c0, implicit=implicit)
        outs = []
        for x in (x0, x1):
            tp = cnn.Tape(params, record=False)
            encs = cnn.encoder(tp, cnn.Var(kf), False, net.running)
            ghat = net.ghat(cnn.coarsest_size(I, True)) if implicit else None
            outs.append(cnn.solver(tp, cnn.Var(x), encs, ghat, False, net.running, True).a)
        return np.abs(outs[1] - outs[0])[0, :, -8:, -8:].max(), np.abs(outs[0]).max()

    d_expl, _ = far_change(Pe, False)
    d_init, _ = far_change(P, True)
    d_long, scale = far_change(P_long, True)
    assert d_expl == 0.0
    assert d_long > 100 * d_init and d_long > 1e3 * np.finfo(float).eps * scale, (d_long, d_init)


def test_composed_preconditioner_reduces_to_its_parts():
    """z = e + V(r - A e) (Section 4.1, multiplicative composition).  A network whose
    output is zero gives exactly the plain V-cycle.  One whose output is the exact error
    A^-1 r leaves nothing for the V-cycle to correct (V(0) = 0), so z = A^-1 r.  For any
    output e, z - e is the V-cycle of the remaining residual."""
    N, abl = 32, 4
    p = hz.Problem(synth.grf_kappa(N - 2 * abl, abl, 4.0, 3), abl)
    V = mg.SLMultigrid(p, 3)
    r = synth.random_complex((N, N), 1)

    class FixedOutput:
        def __init__(self, f):
            self.f = f

        def forward(self, rb, kfeat, train=False):
            return self.f(rb), None

    zero = tr.composed_preconditioner(p, FixedOutput(np.zeros_like), None, V)
    assert np.array_equal(zero(r), V(r))
    assert not np.any(V(np.zeros_like(r)))
    Ad = mg.dense_matrix(p.mass_A)

    def exact(rb):
        return np.stack([np.linalg.solve(Ad, v.ravel()).reshape(N, N) for v in rb])

    e = exact(r[None])[0]
    z = tr.composed_preconditioner(p, FixedOutput(exact), None, V)(r)
    assert np.linalg.norm(z - e) <= 1e-10 * np.linalg.norm(e)
    other = 0.3 * synth.random_complex((1, N, N), 2)
    z = tr.composed_preconditioner(p, FixedOutput(lambda rb: other), None, V)(r)
    assert np.allclose(z - other[0], V(r - p.A(other[0])), rtol=0, atol=1e-13 * np.abs(z).max())


def test_bn_eval_folding_equivalence():
    """Eval-mode BN equals the folded affine a*x + c."""
    rng = np.random.default_rng(3)
    P = {"bn.g": rng.uniform(0.5, 2, 5), "bn.b": rng.standard_normal(5)}
    running = {"bn": (rng.standard_normal(5), rng.uniform(0.5, 2, 5))}
    x = rng.standard_normal((2, 5, 3, 3))
    tp = cnn.Tape(P, record=False)
    y = cnn.batchnorm(tp, cnn.Var(x), "bn", False, running).a
    a, c = cnn.fold_bn(P, running, "bn")
    assert np.allclose(y, a[None, :, None, None] * x + c[None, :, None, None])


def test_eval_forward_is_scale_equivariant_and_zero_safe():
    """Input scaling: e = s Net(r/s) with s = RMS(r), so e(c r) = c e(r) for c > 0."""
    net, P, kf, r, _ = _setup(B=2)
    e1, _ = net.forward(r, kf, train=False)
    e2, _ = net.forward(3.0 * r, kf, train=False)
    assert np.allclose(e2, 3.0 * e1, rtol=1e-12)
    z, _ = net.forward(np.zeros_like(r), kf, train=False)
    assert np.all(np.isfinite(z)) and np.allclose(z, 0.0)


def test_training_pairs_satisfy_r_equals_A_e():
    """Eq. (17): r = b - A x_tilde = A e with e = x - x_tilde."""
    N, abl = 32, 4
    prob = hz.Problem(synth.grf_kappa(N - 2 * abl, abl, 4.0, 2), abl, gamma0=GOLD["train_gamma"]["value"])
    M = mg.SLMultigrid(prob, 3)
    x = synth.smooth_plus_noise(3, N, seed=4)
    k = np.array([2, 5, 20])
    e, r = tr.generate_pairs(prob, M, x, k)
    for i in range(3):
        assert np.allclose(r[i], prob.A(e[i]), atol=1e-12 * np.abs(r[i]).max())
    # more V-cycle iterations leave a smaller residual relative to b = A x
    rel = [np.linalg.norm(r[i]) / np.linalg.norm(prob.A(x[i])) for i in range(3)]
    assert rel[2] < rel[0]
    en, rn = tr.normalise_pairs(e, r)
    assert np.allclose([np.sqrt(np.mean(np.abs(v) ** 2)) for v in rn], 1.0)
    assert np.allclose(rn[1], r[1] / np.sqrt(np.mean(np.abs(r[1]) ** 2)))


def test_mse_loss_gradient_and_adam_first_step():
    rng = np.random.default_rng(5)
    a = rng.standard_normal((3, 4, 4)) + 1j * rng.standard_normal((3, 4, 4))
    b = rng.standard_normal((3, 4, 4)) + 1j * rng.standard_normal((3, 4, 4))
    L, g = tr.mse_loss(a, b)
    assert np.isclose(L, (np.abs(a - b) ** 2).sum() / 3)
    h = 1e-7
    ap = a.copy(); ap[1, 2, 3] += h
    assert np.isclose((tr.mse_loss(ap, b)[0] - L) / h, g[1, 2, 3].real, rtol=1e-5)
    # Adam's first step moves each weight by -lr * sign(g) (bias-corrected moments)
    params = {"w": np.array([1.0, -2.0, 0.5])}
    grads = {"w": np.array([0.3, -4.0, 1e-3])}
    tr.adam_step(params, grads, {}, lr=GOLD["adam_lr"]["value"])
    step = params["w"] - np.array([1.0, -2.0, 0.5])
    assert np.allclose(step, -1e-3 * np.sign(grads["w"]), rtol=1e-4)


@pytest.mark.parametrize("train", [True, False], ids=["train", "eval"])
def test_network_input_gradient_matches_central_differences(train):
    """dL/dr of e = s Net(r / s), s = RMS(r), with the scale's own dependence on r:
    directional derivatives along random complex directions against 4-point central
    differences (FP64), relative 1e-6; and Euler's identity <dL/dr, r> = <dL/de, e>,
    which holds because e is positively homogeneous of degree 1 in r."""
    net, P, kf, r, et = _setup(B=2)
    e, tp = net.forward(r, kf, train=train, skip=True, record=True)
    L, ge = tr.mse_loss(e, et)
    net.backward(tp, ge)
    gr = net.input_gradient(tp, ge)
    assert np.all(np.isfinite(gr))
    rng = np.random.default_rng(11)

    def loss_at(rr):
        running = {k: (v[0].copy(), v[1].copy()) for k, v in net.running.items()}
        saved = net.running
        net.running = running
        ee, _ = net.forward(rr, kf, train=train, skip=True)
        net.running = saved
        return tr.mse_loss(ee, et)[0]

    for _ in range(3):
        d = rng.standard_normal(r.shape) + 1j * rng.standard_normal(r.shape)
        h = 1e-4 * np.abs(r).max()
        vals = [loss_at(r + c * h * d) for c in (2, 1, -1, -2)]
        fd = (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * h)
        an = float(np.real(np.vdot(gr, d)))
        assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-12 * abs(L)), (fd, an)
    euler = float(np.real(np.vdot(gr, r)))
    assert abs(euler - float(np.real(np.vdot(ge, e)))) <= 1e-10 * np.abs(gr).sum() * np.abs(r).max()


def _transposed_params(P):
    """Every 3x3 kernel transposed (convolutions, transposed convolutions, depthwise
    and the implicit kernels); 1x1 weights, biases and BN parameters unchanged."""
    return {k: (np.swapaxes(v, -1, -2).copy() if v.ndim >= 3 and v.shape[-2:] == (3, 3) else v)
            for k, v in P.items()}


@pytest.mark.parametrize("H,W,skip", [(32, 48, True), (32, 64, False)])
@pytest.mark.parametrize("train", [False, True])
def test_rectangular_network_transposes_with_its_kernels(H, W, skip, train):
    """An H x W grid (the out-of-distribution shapes of Section 5.1 are rectangles).
    With every 3x3 kernel transposed, the network maps r^T to e^T: the fixed R and P,
    BatchNorm and softplus commute with the transpose.  A height used for a width
    anywhere on the path (a shape, a crop, an axis of the Green's function) breaks it."""
    c0 = 4
    P = synth.random_params(cnn.param_spec(c0), seed=5, bn_jitter=0.2)
    K = P["s.imp.K"]
    K[:, :, 0, 1] += 0.5          # asymmetric implicit kernels
    net = cnn.Network(P, c0=c0)
    netT = cnn.Network(_transposed_params(P), c0=c0)
    rng = np.random.default_rng(6)
    kf = rng.uniform(0.0625, 1.0, size=(1, 2, H, W))
    r = synth.random_complex((2, H, W), 7)
    e, _ = net.forward(r, kf, train=train, skip=skip)
    assert e.shape == (2, H, W)
    eT, _ = netT.forward(np.swapaxes(r, -1, -2).copy(), np.swapaxes(kf, -1, -2).copy(), train=train, skip=skip)
    assert np.abs(eT - np.swapaxes(e, -1, -2)).max() <= 1e-12 * np.abs(e).max()
    # not a symmetry of the untransposed network: the kernels matter
    e2, _ = net.forward(np.swapaxes(r, -1, -2).copy(), np.swapaxes(kf, -1, -2).copy(), train=train, skip=skip)
    assert np.abs(e2 - np.swapaxes(e, -1, -2)).max() > 1e-3 * np.abs(e).max()


def test_rectangular_coarsest_shape_and_skip_rule():
    """The coarsest map is m_y x m_x (I/16 per axis, or I/8 with the last downsampling
    skipped, Section 5.3); a rectangle skips it when its shorter side is below 512."""
    assert cnn.coarsest_shape(576, 1088) == (36, 68)
    assert cnn.coarsest_shape(448, 896) == (56, 112)
    assert cnn.coarsest_shape(512, 512) == (cnn.coarsest_size(512),) * 2
    assert cnn.coarsest_shape(256, 256) == (cnn.coarsest_size(256),) * 2
