"""Oracle: the encoder-solver U-Net preconditioner network (Sections 4.1-4.4 and 5.3,
Fig. 1), forward and hand-written reverse-mode backward, float64 NCHW.

Test infrastructure only (see the package docstring).

Architecture (c0 = 16, expansion t = 6; readings where the paper is silent):
  Encoder (Section 5.3): input = 2 channels (Re, Im) of kappa^2 (1 - gamma i) at I x I;
    three "downsampling modules" [3x3 stride-2 conv, then two 3x3 convs], each conv
    followed by BatchNorm + softplus (Fig. 1: every convolutional block is);
    outputs enc1 = c0 x I/2, enc2 = 2c0 x I/4, enc3 = 4c0 x I/8.
  Solver (Section 5.3, 4.4):
    r -> s = RMS(r) over the grid, fixed full-weighting R of r/s to I/2 (2 channels)
    level 1: 3x3 conv 2->c0 (stride 1) + BN + softplus, + enc1, inverted bottleneck
    level 2: 3x3 stride-2 conv c0->2c0 + BN + softplus, + enc2, inverted bottleneck
    level 3: 3x3 stride-2 conv 2c0->4c0 + BN + softplus, + enc3, inverted bottleneck
    level 4: downsampling module 4c0->4c0 (first conv stride 2, or stride 1 when
             I < 512, Section 5.3), then the implicit layer on 2c0 complex channels
             (channel k paired with k + 2c0, Section 4.2)
    up 1..3: 3x3 transposed conv (stride 2; stride 1 for up 1 when level 4 kept
             its size) + BN + softplus, two 3x3 convs + BN + softplus, then the
             same-size level output is added (sums, not concatenations, Section 4.4)
    projection: 1x1 conv c0 -> 2 (+ bias), as one complex channel, fixed bilinear P
             to I, times s.
  Inverted bottleneck (MobileNetV2, Section 4.4): 1x1 expand c->tc + BN + softplus,
    3x3 depthwise + BN + softplus, 1x1 project tc->c + BN, identity skip.
  No conv bias where BN follows.  BN eps 1e-5, momentum 0.1; softplus beta = 1.
  Implicit kernels initialised to L + iI (Section 5.3).
  Explicit U-Net (Section 6, the comparison network): the same encoder-solver network
  without the implicit step at the coarsest level (implicit=False below).
  Rectangular grids (the out-of-distribution shapes of Section 5.1; the paper trains on
  squares): an H x W grid runs every layer per axis, the coarsest map is m_y x m_x with
  its Green's function on the per-axis grids, and the last downsampling is skipped when
  the shorter side is below 512.
"""
from __future__ import annotations

import numpy as np
from scipy.special import expit

from . import implicit as imp
from .multigrid import prolong, restrict

BN_EPS = 1e-5
BN_MOMENTUM = 0.1


# ----------------------------------------------------------------------------------
# parameter specification
# ----------------------------------------------------------------------------------

def _conv(spec, name, co, ci, k=3):
    spec.append((name + ".w", (co, ci, k, k), ci * k * k, "w"))


def _convT(spec, name, ci, co):
    # PyTorch ConvTranspose2d layout [Ci, Co, 3, 3]; its default init uses fan_in = Co*9
    spec.append((name + ".w", (ci, co, 3, 3), co * 9, "w"))


def _bn(spec, name, c):
    spec.append((name + ".g", (c,), 0, "bn_g"))
    spec.append((name + ".b", (c,), 0, "bn_b"))


def _ib(spec, name, c, t):
    spec.append((name + ".exp.w", (t * c, c), c, "w"))
    _bn(spec, name + ".bn0", t * c)
    spec.append((name + ".dw.w", (t * c, 3, 3), 9, "w"))
    _bn(spec, name + ".bn1", t * c)
    spec.append((name + ".proj.w", (c, t * c), t * c, "w"))
    _bn(spec, name + ".bn2", c)


def param_spec(c0: int = 16, t: int = 6, implicit: bool = True):
    """Ordered list of (name, shape, fan_in, kind[, values]) for every learnable tensor
    (implicit=False: the explicit U-Net, which has no implicit kernels)."""
    C = [c0, 2 * c0, 4 * c0]
    spec = []
    cin = 2
    for k in range(3):                       # encoder downsampling modules
        _conv(spec, f"e.dm{k+1}.conv0", C[k], cin)
        _bn(spec, f"e.dm{k+1}.bn0", C[k])
        for j in (1, 2):
            _conv(spec, f"e.dm{k+1}.conv{j}", C[k], C[k])
            _bn(spec, f"e.dm{k+1}.bn{j}", C[k])
        cin = C[k]
    cin = 2
    for k in range(3):                       # solver levels 1..3
        _conv(spec, f"s.l{k+1}.conv", C[k], cin)
        _bn(spec, f"s.l{k+1}.bn", C[k])
        _ib(spec, f"s.l{k+1}.ib", C[k], t)
        cin = C[k]
    for j in range(3):                       # level 4 downsampling module
        _conv(spec, f"s.l4.conv{j}", C[2], C[2])
        _bn(spec, f"s.l4.bn{j}", C[2])
    if implicit:
        nk = C[2] // 2                       # implicit layer: complex kernels
        K0 = imp.laplacian_plus_i()
        init = np.stack([np.broadcast_to(K0.real, (nk, 3, 3)), np.broadcast_to(K0.imag, (nk, 3, 3))])
        spec.append(("s.imp.K", (2, nk, 3, 3), 0, "fixed", init.ravel()))
    ups = [(C[2], C[2]), (C[2], C[1]), (C[1], C[0])]
    for k, (ci, co) in enumerate(ups):
        _convT(spec, f"s.up{k+1}.convT", ci, co)
        _bn(spec, f"s.up{k+1}.bn0", co)
        for j in (1, 2):
            _conv(spec, f"s.up{k+1}.conv{j}", co, co)
            _bn(spec, f"s.up{k+1}.bn{j}", co)
    spec.append(("s.proj.w", (2, C[0]), C[0], "w"))
    spec.append(("s.proj.b", (2,), C[0], "bias"))
    return spec


def bn_names(c0: int = 16, t: int = 6):
    """(bn name, channels) for every BatchNorm (running statistics live per name)."""
    out = []
    for name, shape, _, kind, *rest in param_spec(c0, t):
        if kind == "bn_g":
            out.append((name[:-2], shape[0]))
    return out


def init_running(c0: int = 16, t: int = 6):
    return {n: (np.zeros(c), np.ones(c)) for n, c in bn_names(c0, t)}


def num_params(c0: int = 16, t: int = 6, implicit: bool = True) -> int:
    return int(sum(np.prod(s) for _, s, *_ in param_spec(c0, t, implicit)))


# ----------------------------------------------------------------------------------
# a minimal reverse-mode tape
# ----------------------------------------------------------------------------------

class Var:
    __slots__ = ("a", "g")

    def __init__(self, a):
        self.a = a
        self.g = None

    def acc(self, g):
        self.g = g if self.g is None else self.g + g


class Tape:
    def __init__(self, params, grads=None, record=True):
        self.params = params
        self.grads = {} if grads is None else grads
        self.record = record
        self.ops = []

    def push(self, fn):
        if self.record:
            self.ops.append(fn)

    def pgrad(self, name, g):
        self.grads[name] = self.grads.get(name, 0.0) + g

    def backward(self):
        for fn in reversed(self.ops):
            fn()


def _pad1(x):
    return np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))


# --- 3x3 convolution (cross-correlation), zero padding 1 ----------------------------

def conv3x3(tp: Tape, x: Var, wname: str, stride: int) -> Var:
    w = tp.params[wname]
    B, Ci, H, W = x.a.shape
    Ho, Wo = (H - 1) // stride + 1, (W - 1) // stride + 1
    xp = _pad1(x.a)
    sl = lambda ky, kx: (slice(None), slice(None),
                         slice(ky, ky + stride * (Ho - 1) + 1, stride),
                         slice(kx, kx + stride * (Wo - 1) + 1, stride))
    y = np.zeros((B, w.shape[0], Ho, Wo))
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("oc,bchw->bohw", w[:, :, ky, kx], xp[sl(ky, kx)])
    out = Var(y)

    def bwd():
        dxp = np.zeros_like(xp)
        dw = np.zeros_like(w)
        for ky in range(3):
            for kx in range(3):
                dw[:, :, ky, kx] = np.einsum("bohw,bchw->oc", out.g, xp[sl(ky, kx)])
                dxp[sl(ky, kx)] += np.einsum("oc,bohw->bchw", w[:, :, ky, kx], out.g)
        tp.pgrad(wname, dw)
        x.acc(dxp[:, :, 1:-1, 1:-1])
    tp.push(bwd)
    return out


def conv3x3_transposed(tp: Tape, x: Var, wname: str, stride: int) -> Var:
    """Transposed 3x3 convolution, padding 1, output size stride*H (output padding
    stride-1): full[s*y+ky, s*x+kx] += sum_ci w[ci,co,ky,kx] x[ci,y,x], cropped at 1."""
    w = tp.params[wname]
    B, Ci, H, W = x.a.shape
    s = stride
    full = np.zeros((B, w.shape[1], s * (H - 1) + 3 + (s - 1), s * (W - 1) + 3 + (s - 1)))
    sl = lambda ky, kx: (slice(None), slice(None),
                         slice(ky, ky + s * (H - 1) + 1, s), slice(kx, kx + s * (W - 1) + 1, s))
    for ky in range(3):
        for kx in range(3):
            full[sl(ky, kx)] += np.einsum("co,bchw->bohw", w[:, :, ky, kx], x.a)
    out = Var(full[:, :, 1:1 + s * H, 1:1 + s * W].copy())

    def bwd():
        dfull = np.zeros_like(full)
        dfull[:, :, 1:1 + s * H, 1:1 + s * W] = out.g
        dx = np.zeros_like(x.a)
        dw = np.zeros_like(w)
        for ky in range(3):
            for kx in range(3):
                dx += np.einsum("co,bohw->bchw", w[:, :, ky, kx], dfull[sl(ky, kx)])
                dw[:, :, ky, kx] = np.einsum("bchw,bohw->co", x.a, dfull[sl(ky, kx)])
        tp.pgrad(wname, dw)
        x.acc(dx)
    tp.push(bwd)
    return out


def conv1x1(tp: Tape, x: Var, wname: str, bname: str | None = None) -> Var:
    w = tp.params[wname]
    y = np.einsum("oc,bchw->bohw", w, x.a)
    if bname is not None:
        y = y + tp.params[bname][None, :, None, None]
    out = Var(y)

    def bwd():
        tp.pgrad(wname, np.einsum("bohw,bchw->oc", out.g, x.a))
        if bname is not None:
            tp.pgrad(bname, out.g.sum(axis=(0, 2, 3)))
        x.acc(np.einsum("oc,bohw->bchw", w, out.g))
    tp.push(bwd)
    return out


def depthwise3x3(tp: Tape, x: Var, wname: str) -> Var:
    w = tp.params[wname]
    B, C, H, W = x.a.shape
    xp = _pad1(x.a)
    y = np.zeros_like(x.a)
    for ky in range(3):
        for kx in range(3):
            y += w[None, :, ky, kx, None, None] * xp[:, :, ky:ky + H, kx:kx + W]
    out = Var(y)

    def bwd():
        dxp = np.zeros_like(xp)
        dw = np.zeros_like(w)
        for ky in range(3):
            for kx in range(3):
                dw[:, ky, kx] = np.einsum("bchw,bchw->c", out.g, xp[:, :, ky:ky + H, kx:kx + W])
                dxp[:, :, ky:ky + H, kx:kx + W] += w[None, :, ky, kx, None, None] * out.g
        tp.pgrad(wname, dw)
        x.acc(dxp[:, :, 1:-1, 1:-1])
    tp.push(bwd)
    return out


def batchnorm(tp: Tape, x: Var, name: str, train: bool, running: dict) -> Var:
    """BatchNorm2d: batch statistics (biased variance) in training, running
    statistics in evaluation; running stats updated with momentum 0.1 and the
    unbiased batch variance."""
    g, b = tp.params[name + ".g"], tp.params[name + ".b"]
    if train:
        mu = x.a.mean(axis=(0, 2, 3))
        var = x.a.var(axis=(0, 2, 3))
        n = x.a.size // x.a.shape[1]
        if running is not None:
            rm, rv = running[name]
            running[name] = ((1 - BN_MOMENTUM) * rm + BN_MOMENTUM * mu,
                             (1 - BN_MOMENTUM) * rv + BN_MOMENTUM * var * n / max(n - 1, 1))
    else:
        mu, var = running[name]
    inv = 1.0 / np.sqrt(var + BN_EPS)
    xh = (x.a - mu[None, :, None, None]) * inv[None, :, None, None]
    out = Var(g[None, :, None, None] * xh + b[None, :, None, None])

    def bwd():
        dy = out.g
        tp.pgrad(name + ".g", (dy * xh).sum(axis=(0, 2, 3)))
        tp.pgrad(name + ".b", dy.sum(axis=(0, 2, 3)))
        dxh = dy * g[None, :, None, None]
        if train:
            n = dy.size // dy.shape[1]
            s1 = dxh.sum(axis=(0, 2, 3))[None, :, None, None]
            s2 = (dxh * xh).sum(axis=(0, 2, 3))[None, :, None, None]
            x.acc(inv[None, :, None, None] * (dxh - s1 / n - xh * s2 / n))
        else:
            x.acc(dxh * inv[None, :, None, None])
    tp.push(bwd)
    return out


def softplus(tp: Tape, x: Var) -> Var:
    out = Var(np.logaddexp(0.0, x.a))

    def bwd():
        x.acc(out.g * expit(x.a))
    tp.push(bwd)
    return out


def add(tp: Tape, x: Var, y: Var) -> Var:
    """x + y; if y has fewer batch entries (G dividing B), entry g is added to the g-th
    group of B/G consecutive samples (each slowness model's encoding feeds the samples
    drawn for it; G = 1 is a plain broadcast)."""
    B, G = x.a.shape[0], y.a.shape[0]
    rep = B // G
    out = Var(x.a + np.repeat(y.a, rep, axis=0))

    def bwd():
        x.acc(out.g)
        y.acc(out.g.reshape((G, rep) + out.g.shape[1:]).sum(axis=1))
    tp.push(bwd)
    return out


def implicit_layer(tp: Tape, x: Var, kname: str, ghat: np.ndarray) -> Var:
    """Eq. (14) on channel pairs (k, k + C/2) read as complex channels; `ghat`
    [C/2, 2m, 2m] was built from the kernels by Eq. (15)."""
    C = x.a.shape[1]
    nk = C // 2
    z = x.a[:, :nk] + 1j * x.a[:, nk:]
    y = np.stack([imp.implicit_apply(z[:, k], ghat[k]) for k in range(nk)], axis=1)
    out = Var(np.concatenate([y.real, y.imag], axis=1))

    def bwd():
        gy = out.g[:, :nk] + 1j * out.g[:, nk:]
        gx = np.stack([imp.implicit_adjoint(gy[:, k], ghat[k]) for k in range(nk)], axis=1)
        x.acc(np.concatenate([gx.real, gx.imag], axis=1))
        m = x.a.shape[-2:]
        K = tp.params[kname]
        gK = np.zeros_like(K)
        for k in range(nk):
            g_gh = imp.implicit_grad_ghat(z[:, k], gy[:, k])
            gk = imp.greens_backward(K[0, k] + 1j * K[1, k], m, g_gh)
            gK[0, k] = gk.real
            gK[1, k] = gk.imag
        tp.pgrad(kname, gK)
    tp.push(bwd)
    return out


# ----------------------------------------------------------------------------------
# network
# ----------------------------------------------------------------------------------

def skip_last_down(I: int, threshold: int = 512) -> bool:
    """Section 5.3: below 512 x 512 the last downsampling is skipped."""
    return I < threshold


def coarsest_size(I: int, skip: bool | None = None) -> int:
    skip = skip_last_down(I) if skip is None else skip
    return I // 8 if skip else I // 16


def coarsest_shape(H: int, W: int, skip: bool | None = None) -> tuple[int, int]:
    """(m_y, m_x) of an H x W grid.  The paper's grids are square; on a rectangle the
    last downsampling is skipped when the shorter side is below the threshold."""
    skip = skip_last_down(min(H, W)) if skip is None else skip
    return coarsest_size(H, skip), coarsest_size(W, skip)


def build_ghat(params, m: int, literal: bool = False) -> np.ndarray:
    K = params["s.imp.K"]
    return np.stack([imp.greens_hat(K[0, k] + 1j * K[1, k], m, literal=literal)
                     for k in range(K.shape[1])])


def conv_bn_act(tp, x, cname, bname, stride, train, running, transposed=False):
    z = (conv3x3_transposed if transposed else conv3x3)(tp, x, cname + ".w", stride)
    return softplus(tp, batchnorm(tp, z, bname, train, running))


def inverted_bottleneck(tp, x, name, train, running):
    a = softplus(tp, batchnorm(tp, conv1x1(tp, x, name + ".exp.w"), name + ".bn0", train, running))
    a = softplus(tp, batchnorm(tp, depthwise3x3(tp, a, name + ".dw.w"), name + ".bn1", train, running))
    a = batchnorm(tp, conv1x1(tp, a, name + ".proj.w"), name + ".bn2", train, running)
    return add(tp, x, a)


def encoder(tp, kfeat: Var, train, running):
    """kfeat [Bk, 2, I, I] -> [enc1, enc2, enc3]."""
    x = kfeat
    outs = []
    for k in range(3):
        p = f"e.dm{k+1}"
        x = conv_bn_act(tp, x, p + ".conv0", p + ".bn0", 2, train, running)
        x = conv_bn_act(tp, x, p + ".conv1", p + ".bn1", 1, train, running)
        x = conv_bn_act(tp, x, p + ".conv2", p + ".bn2", 1, train, running)
        outs.append(x)
    return outs


def solver(tp, x0: Var, encs, ghat, train, running, skip: bool):
    """x0 [B, 2, I/2, I/2] (restricted, normalised residual) -> p [B, 2, I/2, I/2];
    ghat None: the explicit U-Net (no implicit step)."""
    feats = []
    x = x0
    for k in range(3):
        p = f"s.l{k+1}"
        x = conv_bn_act(tp, x, p + ".conv", p + ".bn", 1 if k == 0 else 2, train, running)
        x = add(tp, x, encs[k])
        x = inverted_bottleneck(tp, x, p + ".ib", train, running)
        feats.append(x)
    x = conv_bn_act(tp, x, "s.l4.conv0", "s.l4.bn0", 1 if skip else 2, train, running)
    x = conv_bn_act(tp, x, "s.l4.conv1", "s.l4.bn1", 1, train, running)
    x = conv_bn_act(tp, x, "s.l4.conv2", "s.l4.bn2", 1, train, running)
    if ghat is not None:
        x = implicit_layer(tp, x, "s.imp.K", ghat)
    for k in range(3):
        p = f"s.up{k+1}"
        st = 1 if (k == 0 and skip) else 2
        x = conv_bn_act(tp, x, p + ".convT", p + ".bn0", st, train, running, transposed=True)
        x = conv_bn_act(tp, x, p + ".conv1", p + ".bn1", 1, train, running)
        x = conv_bn_act(tp, x, p + ".conv2", p + ".bn2", 1, train, running)
        x = add(tp, x, feats[2 - k])
    return conv1x1(tp, x, "s.proj.w", "s.proj.b")


def kappa_features(kappa: np.ndarray, gamma: np.ndarray) -> np.ndarray:
    """Encoder input: (Re, Im) of kappa^2 (1 - gamma i) as [1, 2, N, N]."""
    k2 = kappa.astype(np.float64) ** 2
    return np.stack([k2, -k2 * gamma])[None]


class Network:
    """Encoder-solver network with parameters `params` (dict name -> float64 array)
    and BatchNorm running statistics `running` (dict bn name -> (mean, var));
    implicit=False is the explicit U-Net of Section 6."""

    def __init__(self, params, running=None, c0: int = 16, t: int = 6, literal_green=False,
                 implicit: bool = True):
        self.params = params
        self.c0, self.t = c0, t
        self.implicit = implicit
        self.running = init_running(c0, t) if running is None else running
        self.literal_green = literal_green
        self._ghat = {}

    def ghat(self, m: int):
        return build_ghat(self.params, m, self.literal_green)

    def forward(self, r: np.ndarray, kfeat: np.ndarray, train: bool = False,
                skip: bool | None = None, record: bool = False):
        """e = s * Net(r / s), s = RMS of r over the grid, for a batch r [B, H, W] complex
        (the paper leaves the scale unstated; the RMS is this implementation's choice).
        The paper's grids are square (H = W); a rectangle runs every layer per axis.

        Returns (e, tape, scale); the tape's backward accumulates parameter
        gradients in tape.grads given the complex gradient of the loss w.r.t. e.
        """
        B, H, W = r.shape
        skip = skip_last_down(min(H, W)) if skip is None else skip
        # s is the residual's RMS over the grid, so the network sees O(1)
        # values at every grid size (the multiscale setting of Section 4.3)
        s = np.sqrt((np.abs(r) ** 2).reshape(B, -1).mean(axis=1))
        s_safe = np.where(s > 0, s, 1.0)
        rn = r / s_safe[:, None, None]
        rc = restrict(rn)                                     # fixed R to I/2
        x0 = Var(np.stack([rc.real, rc.imag], axis=1))
        tp = Tape(self.params, record=record)
        tp.x0, tp.r, tp.s_safe = x0, r, s_safe
        running = self.running if train else self.running
        kf = Var(kfeat)
        encs = encoder(tp, kf, train, running)
        m = coarsest_shape(H, W, skip)
        if m[0] == m[1]:
            m = m[0]
        p = solver(tp, x0, encs, self.ghat(m) if self.implicit else None, train, running, skip)
        pc = p.a[:, 0] + 1j * p.a[:, 1]
        e = prolong(pc) * s[:, None, None]
        tp.out = p
        tp.scale = s
        tp.e = e
        return e, tp

    def backward(self, tp: Tape, grad_e: np.ndarray):
        """Back-propagate the complex gradient grad_e (dL/dRe e + i dL/dIm e)."""
        s = tp.scale
        gpc = 4.0 * restrict(grad_e) * s[:, None, None]       # P^T = 4 R
        tp.out.g = np.stack([gpc.real, gpc.imag], axis=1)
        tp.backward()
        return tp.grads

    def input_gradient(self, tp: Tape, grad_e: np.ndarray) -> np.ndarray:
        """dL/dRe r + i dL/dIm r after `backward(tp, grad_e)`, through every step of
        e = s P(Net(R(r / s))), s = RMS(r) = sqrt(<r, r> / n) (n grid points per
        sample, <a, b> = Re sum conj(a) b), the scale included:
            u = r / s                 ->  dL/du = R^T dL/dx0 = P(dL/dx0) / 4
            e = s q, q = P(Net(R u))  ->  dL/ds (direct) = <grad_e, q>
            u = r / s                 ->  dL/dr = dL/du / s,  dL/ds -= <dL/du, r> / s^2
            s = sqrt(<r, r> / n)      ->  dL/dr += dL/ds r / (n s)
        A zero sample (s = 0) gets a zero gradient."""
        gx = tp.x0.g
        gu = prolong(gx[:, 0] + 1j * gx[:, 1]) / 4.0
        r, s, e = tp.r, tp.scale, tp.e
        B = r.shape[0]
        n = r[0].size
        out = np.zeros_like(r)
        for b in range(B):
            if not s[b] > 0:
                continue
            q = e[b] / s[b]
            gs = np.real(np.vdot(grad_e[b], q)) - np.real(np.vdot(gu[b], r[b])) / s[b] ** 2
            out[b] = gu[b] / s[b] + gs * r[b] / (n * s[b])
        return out


def fold_bn(params, running, name):
    """Eval-mode BatchNorm as a per-channel affine map y = a x + c."""
    g, b = params[name + ".g"], params[name + ".b"]
    mu, var = running[name]
    a = g / np.sqrt(var + BN_EPS)
    return a, b - mu * a
