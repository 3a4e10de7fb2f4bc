"""Pins of the oracle network's forward layers (Sections 4.4 and 5.3: 3x3 convolutions
at stride 1 and 2, the transposed stride-2 convolution of the up path, the depthwise
3x3 and the 1x1 convolutions of the inverted bottleneck, training- and
evaluation-mode BatchNorm, softplus) against definitions that do not go through the
oracle (no GPU).

The paper builds its network from PyTorch modules (Section 3.4), so those modules'
conventions define what each layer computes: cross-correlation (no kernel flip),
zero padding 1, the transposed convolution as the adjoint of the strided one with
output padding 1, BatchNorm normalising with the biased batch variance and updating
its running variance with the unbiased one.  Each layer is checked two ways:
against SciPy's 2-D correlation or a hand-worked example, and against the PyTorch
CPU module itself in float64.  A flipped kernel, a one-pixel offset, a missing
output-padding row or a swapped variance would fail here, whereas the
finite-difference tests, which check backward against forward, would not see them.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F
from scipy.signal import correlate2d

from oracle import cnn


def _rng(seed):
    return np.random.default_rng(seed)


def _run(layer, x, params, **kw):
    tp = cnn.Tape(params, record=False)
    return layer(tp, cnn.Var(x), **kw).a


@pytest.mark.parametrize("H,W", [(7, 9), (8, 8), (5, 12)])
def test_conv3x3_stride1_is_zero_padded_cross_correlation(H, W):
    """y[o] = sum_c correlate(x[c], w[o, c]) with zero padding 1 (no kernel flip)."""
    rng = _rng(H * W)
    B, Ci, Co = 2, 3, 4
    x = rng.standard_normal((B, Ci, H, W))
    w = rng.standard_normal((Co, Ci, 3, 3))
    y = _run(cnn.conv3x3, x, {"c.w": w}, wname="c.w", stride=1)
    ref = np.zeros((B, Co, H, W))
    for b in range(B):
        for o in range(Co):
            for c in range(Ci):
                ref[b, o] += correlate2d(x[b, c], w[o, c], mode="same", boundary="fill", fillvalue=0.0)
    assert y.shape == ref.shape
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
    tref = F.conv2d(torch.from_numpy(x), torch.from_numpy(w), stride=1, padding=1).numpy()
    assert np.abs(y - tref).max() <= 1e-13 * np.abs(tref).max()


@pytest.mark.parametrize("H,W", [(8, 8), (7, 10), (9, 5)])
def test_conv3x3_stride2_samples_the_stride1_correlation_at_even_points(H, W):
    """Stride 2, padding 1: output (ceil(H/2), ceil(W/2)) with y[i, j] equal to the
    zero-padded correlation centred on input (2i, 2j)."""
    rng = _rng(H + 17 * W)
    B, Ci, Co = 2, 3, 2
    x = rng.standard_normal((B, Ci, H, W))
    w = rng.standard_normal((Co, Ci, 3, 3))
    y = _run(cnn.conv3x3, x, {"c.w": w}, wname="c.w", stride=2)
    assert y.shape == (B, Co, (H + 1) // 2, (W + 1) // 2)
    full = np.zeros((B, Co, H, W))
    for b in range(B):
        for o in range(Co):
            for c in range(Ci):
                full[b, o] += correlate2d(x[b, c], w[o, c], mode="same", boundary="fill", fillvalue=0.0)
    assert np.abs(y - full[:, :, ::2, ::2]).max() <= 1e-13 * np.abs(full).max()
    tref = F.conv2d(torch.from_numpy(x), torch.from_numpy(w), stride=2, padding=1).numpy()
    assert np.abs(y - tref).max() <= 1e-13 * np.abs(tref).max()


@pytest.mark.parametrize("H,W", [(4, 4), (3, 5), (6, 2)])
def test_transposed_stride2_conv_is_the_adjoint_of_the_strided_conv(H, W):
    """The up path's 3x3 transposed convolution (stride 2, padding 1, output padding 1)
    with weights w [Ci, Co, 3, 3] is the adjoint of the stride-2 convolution with the
    same tensor read as [out = Ci][in = Co]: <T x, y> = <x, C y> for every x (H x W)
    and y (2H x 2W), and its output is exactly 2H x 2W."""
    rng = _rng(31 * H + W)
    B, Ci, Co = 2, 3, 4
    w = rng.standard_normal((Ci, Co, 3, 3))
    x = rng.standard_normal((B, Ci, H, W))
    yb = rng.standard_normal((B, Co, 2 * H, 2 * W))
    Tx = _run(cnn.conv3x3_transposed, x, {"t.w": w}, wname="t.w", stride=2)
    assert Tx.shape == (B, Co, 2 * H, 2 * W)
    Cy = _run(cnn.conv3x3, yb, {"t.w": w}, wname="t.w", stride=2)
    assert Cy.shape == x.shape
    lhs, rhs = float((Tx * yb).sum()), float((x * Cy).sum())
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(Tx).sum() * np.abs(yb).max())
    # the adjoint identity fixes T completely; PyTorch's module agrees
    tref = F.conv_transpose2d(torch.from_numpy(x), torch.from_numpy(w), stride=2, padding=1,
                              output_padding=1).numpy()
    assert np.abs(Tx - tref).max() <= 1e-13 * np.abs(tref).max()
    # brute force from the definition: every input pixel scatters w into the output
    # grid around (2i, 2j), positions outside 0..2H-1 / 0..2W-1 dropped
    ref = np.zeros_like(Tx)
    for b in range(B):
        for c in range(Ci):
            for i in range(H):
                for j in range(W):
                    for ky in range(3):
                        for kx in range(3):
                            oy, ox = 2 * i + ky - 1, 2 * j + kx - 1
                            if 0 <= oy < 2 * H and 0 <= ox < 2 * W:
                                ref[b, :, oy, ox] += w[c, :, ky, kx] * x[b, c, i, j]
    assert np.abs(Tx - ref).max() <= 1e-13 * np.abs(ref).max()


def test_transposed_stride1_conv_is_the_flipped_correlation():
    """The first up module at grids that keep the coarsest size uses a stride-1
    transposed conv: the correlation with the 180-degree-rotated kernel and swapped
    channel roles."""
    rng = _rng(5)
    B, Ci, Co, H, W = 2, 3, 2, 6, 7
    w = rng.standard_normal((Ci, Co, 3, 3))
    x = rng.standard_normal((B, Ci, H, W))
    y = _run(cnn.conv3x3_transposed, x, {"t.w": w}, wname="t.w", stride=1)
    wf = np.ascontiguousarray(np.transpose(w[:, :, ::-1, ::-1], (1, 0, 2, 3)))
    ref = _run(cnn.conv3x3, x, {"c.w": wf}, wname="c.w", stride=1)
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
    tref = F.conv_transpose2d(torch.from_numpy(x), torch.from_numpy(w), stride=1, padding=1).numpy()
    assert np.abs(y - tref).max() <= 1e-13 * np.abs(tref).max()


def test_depthwise3x3_is_a_per_channel_correlation():
    rng = _rng(9)
    B, C, H, W = 2, 5, 6, 9
    x = rng.standard_normal((B, C, H, W))
    w = rng.standard_normal((C, 3, 3))
    y = _run(cnn.depthwise3x3, x, {"d.w": w}, wname="d.w")
    for b in range(B):
        for c in range(C):
            ref = correlate2d(x[b, c], w[c], mode="same", boundary="fill", fillvalue=0.0)
            assert np.abs(y[b, c] - ref).max() <= 1e-13 * np.abs(ref).max()
    tref = F.conv2d(torch.from_numpy(x), torch.from_numpy(w[:, None]), padding=1, groups=C).numpy()
    assert np.abs(y - tref).max() <= 1e-13 * np.abs(tref).max()


def test_conv1x1_with_bias_is_a_channel_matrix_product():
    rng = _rng(12)
    x = rng.standard_normal((2, 4, 3, 5))
    w = rng.standard_normal((3, 4))
    bias = rng.standard_normal(3)
    y = _run(cnn.conv1x1, x, {"p.w": w, "p.b": bias}, wname="p.w", bname="p.b")
    ref = np.zeros((2, 3, 3, 5))
    for o in range(3):
        ref[:, o] = bias[o] + sum(w[o, c] * x[:, c] for c in range(4))
    assert np.abs(y - ref).max() <= 1e-14 * np.abs(ref).max()


def test_batchnorm_training_mode_on_a_hand_worked_example():
    """One channel holding 1, 2, 3, 4 (batch 2 x 1 x 2 pixels): batch mean 2.5, biased
    variance 1.25 normalises; the running statistics move by momentum 0.1 toward the
    mean and the UNBIASED variance 5/3."""
    x = np.array([1.0, 2.0, 3.0, 4.0]).reshape(2, 1, 1, 2)
    params = {"bn.g": np.array([2.0]), "bn.b": np.array([0.5])}
    running = {"bn": (np.array([0.0]), np.array([1.0]))}
    y = _run(cnn.batchnorm, x, params, name="bn", train=True, running=running)
    expect = 2.0 * (np.array([1.0, 2.0, 3.0, 4.0]) - 2.5) / np.sqrt(1.25 + 1e-5) + 0.5
    assert np.abs(y.ravel() - expect).max() <= 1e-14
    rm, rv = running["bn"]
    assert abs(rm[0] - 0.25) <= 1e-15
    assert abs(rv[0] - (0.9 + 0.1 * 5.0 / 3.0)) <= 1e-15


@pytest.mark.parametrize("train", [True, False], ids=["train", "eval"])
def test_batchnorm_matches_the_pytorch_module(train):
    rng = _rng(21)
    C = 6
    x = rng.standard_normal((3, C, 4, 5)) * rng.uniform(0.5, 3, C)[None, :, None, None] + 2.0
    g, b = rng.uniform(0.5, 2, C), rng.standard_normal(C)
    rm0, rv0 = rng.standard_normal(C), rng.uniform(0.5, 2, C)
    running = {"bn": (rm0.copy(), rv0.copy())}
    y = _run(cnn.batchnorm, x, {"bn.g": g, "bn.b": b}, name="bn", train=train, running=running)
    trm, trv = torch.from_numpy(rm0.copy()), torch.from_numpy(rv0.copy())
    ty = F.batch_norm(torch.from_numpy(x), trm, trv, torch.from_numpy(g), torch.from_numpy(b), training=train,
                      momentum=cnn.BN_MOMENTUM, eps=cnn.BN_EPS).numpy()
    assert np.abs(y - ty).max() <= 1e-12 * np.abs(ty).max()
    assert np.abs(running["bn"][0] - trm.numpy()).max() <= 1e-14
    assert np.abs(running["bn"][1] - trv.numpy()).max() <= 1e-14


def test_softplus_matches_its_definition_without_overflow():
    x = np.array([-800.0, -30.0, -1.0, 0.0, 0.5, 30.0, 800.0])
    tp = cnn.Tape({}, record=False)
    y = cnn.softplus(tp, cnn.Var(x)).a
    assert np.all(np.isfinite(y))
    mid = np.abs(x) < 40
    assert np.allclose(y[mid], np.log1p(np.exp(x[mid])), rtol=1e-15, atol=0)
    assert y[0] == 0.0 and y[-1] == 800.0
    # PyTorch returns x itself above x = 20, where log(1 + e^-x) < 3e-9 relative
    assert np.allclose(y, F.softplus(torch.from_numpy(x)).numpy(), rtol=1e-13, atol=0)


@pytest.mark.parametrize("train", [True, False], ids=["train", "eval"])
def test_inverted_bottleneck_matches_the_pytorch_module_chain(train):
    """The MobileNetV2 block of Section 4.4 (1x1 expand, BN, softplus, depthwise 3x3,
    BN, softplus, 1x1 project, BN, identity skip), composed from PyTorch modules."""
    rng = _rng(33)
    C, t, B, H, W = 4, 6, 2, 5, 7
    E = t * C
    P = {"ib.exp.w": rng.standard_normal((E, C)) * 0.5, "ib.dw.w": rng.standard_normal((E, 3, 3)) * 0.5,
         "ib.proj.w": rng.standard_normal((C, E)) * 0.3}
    running = {}
    for nm, c in (("ib.bn0", E), ("ib.bn1", E), ("ib.bn2", C)):
        P[nm + ".g"], P[nm + ".b"] = rng.uniform(0.5, 1.5, c), 0.2 * rng.standard_normal(c)
        running[nm] = (0.3 * rng.standard_normal(c), rng.uniform(0.5, 2, c))
    x = rng.standard_normal((B, C, H, W))
    run0 = {k: (v[0].copy(), v[1].copy()) for k, v in running.items()}
    tp = cnn.Tape(P, record=False)
    y = cnn.inverted_bottleneck(tp, cnn.Var(x), "ib", train, running).a

    T = lambda a: torch.from_numpy(np.ascontiguousarray(a))
    tr_run = {k: (T(v[0]), T(v[1])) for k, v in run0.items()}

    def bn(z, nm):
        return F.batch_norm(z, tr_run[nm][0], tr_run[nm][1], T(P[nm + ".g"]), T(P[nm + ".b"]), training=train,
                            momentum=cnn.BN_MOMENTUM, eps=cnn.BN_EPS)

    z = F.softplus(bn(F.conv2d(T(x), T(P["ib.exp.w"][:, :, None, None])), "ib.bn0"))
    z = F.softplus(bn(F.conv2d(z, T(P["ib.dw.w"][:, None]), padding=1, groups=E), "ib.bn1"))
    z = bn(F.conv2d(z, T(P["ib.proj.w"][:, :, None, None])), "ib.bn2")
    ty = (T(x) + z).numpy()
    assert np.abs(y - ty).max() <= 1e-12 * np.abs(ty).max()
    for nm in running:
        assert np.abs(running[nm][0] - tr_run[nm][0].numpy()).max() <= 1e-13
        assert np.abs(running[nm][1] - tr_run[nm][1].numpy()).max() <= 1e-13
