"""Oracle: training data generation (Eq. 17), the MSE loss (Eq. 16), the composed
preconditioner (Section 4.1) and the Adam update (Section 5.3).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from .fgmres import fgmres


def generate_pairs(problem, vcycle, x: np.ndarray, iters: np.ndarray):
    """Eq. (17): b = A x; x_tilde = FGMRES(A, M = V-cycle, b, x0 = 0) run for exactly
    iters[i] iterations (one cycle, restart >= iters[i]); e = x - x_tilde,
    r = b - A x_tilde.  x [B, N, N] complex; returns (e, r)."""
    e = np.empty_like(x)
    r = np.empty_like(x)
    for i in range(x.shape[0]):
        b = problem.A(x[i])
        k = int(iters[i])
        xt, _ = fgmres(problem.A, b, np.zeros_like(b), vcycle, restart=k, tol=0.0, maxit=k)
        e[i] = x[i] - xt
        r[i] = b - problem.A(xt)
    return e, r


def normalise_pairs(e: np.ndarray, r: np.ndarray):
    """The paper leaves the input scale unstated; here training pairs are scaled by 1/s_i (both e and r), s_i the RMS of
    r_i over the grid."""
    s = np.sqrt((np.abs(r) ** 2).reshape(r.shape[0], -1).mean(axis=1))
    return e / s[:, None, None], r / s[:, None, None]


def mse_loss(e_pred: np.ndarray, e_true: np.ndarray):
    """Eq. (16): (1/m) sum_i ||e_pred_i - e_true_i||_2^2 over all real components.
    Returns (loss, complex gradient dL/dRe + i dL/dIm)."""
    m = e_pred.shape[0]
    d = e_pred - e_true
    return float((np.abs(d) ** 2).sum() / m), 2.0 * d / m


def composed_preconditioner(problem, net, kfeat, vcycle):
    """Section 4.1: the network maps a residual to an error, which a V-cycle then
    smooths.  Read as a multiplicative composition: z = e + V(r - A e), e = Net(r)."""
    def M(r):
        rb = r[None] if r.ndim == 2 else r
        e, _ = net.forward(rb, kfeat, train=False)
        z = e + vcycle(rb - problem.A(e))
        return z[0] if r.ndim == 2 else z
    return M


def adam_step(params: dict, grads: dict, state: dict, lr: float, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma & Ba, default hyper-parameters as in Section 5.3)."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for k, g in grads.items():
        m, v = state.get(("m", k), 0.0), state.get(("v", k), 0.0)
        m = beta1 * m + (1 - beta1) * g
        v = beta2 * v + (1 - beta2) * g * g
        state[("m", k)], state[("v", k)] = m, v
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
