"""Oracle: flexible GMRES (Saad 1993, cited in Section 1 as the Krylov method the
preconditioners run in), right-preconditioned and restarted.

Test infrastructure only (see the package docstring).

Conventions: <u, v> = sum conj(u) v; modified Gram-Schmidt Arnoldi; complex Givens
rotations; relative residual ||b - A x|| / ||b|| against the original b; the
iteration count is the number of Arnoldi steps (one preconditioner application
each).  A step whose Givens residual estimate drops below tol ends the cycle; the
true residual then decides convergence.
"""
from __future__ import annotations

import numpy as np


def givens(a: complex, b: complex):
    """Complex Givens rotation [[c, s], [-conj(s), c]] (c real) that maps (a, b) to (r, 0)."""
    if a == 0:
        return 0.0, 1.0 + 0j, b
    t = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    c = abs(a) / t
    s = (a / abs(a)) * np.conj(b) / t
    return c, s, (a / abs(a)) * t


class FGMRESResult:
    def __init__(self):
        self.iters = 0
        self.converged = False
        self.res_hist = []   # true relative residual after every cycle
        self.est_hist = []   # Givens estimate after every Arnoldi step
        self.V = None        # last cycle's basis (for Arnoldi-relation tests)
        self.Z = None
        self.H = None


def fgmres(A, b: np.ndarray, x0: np.ndarray, M, restart: int, tol: float, maxit: int,
           bnorm: float | None = None, keep_basis: bool = False):
    """Right-preconditioned flexible GMRES(restart).

    A, M   : callables on arrays shaped like b (M may change from call to call)
    tol    : stop when ||b - A x|| <= tol * bnorm (bnorm defaults to ||b||)
    maxit  : cap on the total number of Arnoldi steps
    Returns (x, FGMRESResult).
    """
    res = FGMRESResult()
    bnorm = np.linalg.norm(b) if bnorm is None else bnorm
    x = np.array(x0, dtype=np.complex128, copy=True)
    if bnorm == 0.0:
        res.converged = True
        return np.zeros_like(x), res
    r = b - A(x)
    beta = np.linalg.norm(r)
    res.res_hist.append(beta / bnorm)
    if beta <= tol * bnorm:
        res.converged = True
        return x, res
    while res.iters < maxit:
        m = min(restart, maxit - res.iters)
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        k = 0
        breakdown = False
        for j in range(m):
            z = M(V[j])
            Z.append(z)
            w = A(z)
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            res.iters += 1
            k = j + 1
            if H[j + 1, j] == 0.0:
                breakdown = True
            else:
                V.append(w / H[j + 1, j])
            # apply previous rotations to column j, then a new one
            for i in range(j):
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hi1
                H[i + 1, j] = -np.conj(sn[i]) * hi + cs[i] * hi1
            cs[j], sn[j], H[j, j] = givens(H[j, j], H[j + 1, j])
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            res.est_hist.append(abs(g[j + 1]) / bnorm)
            if breakdown or abs(g[j + 1]) <= tol * bnorm:
                break
        # back substitution with the rotated (upper-triangular) H
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        for i in range(k):
            x = x + y[i] * Z[i]
        if keep_basis:
            res.V, res.Z = V, Z
        r = b - A(x)
        beta = np.linalg.norm(r)
        res.res_hist.append(beta / bnorm)
        if beta <= tol * bnorm or breakdown:
            res.converged = beta <= tol * bnorm
            break
    return x, res


def arnoldi_flexible(A, M, r0: np.ndarray, m: int):
    """m steps of flexible Arnoldi with MGS, returning (V [m+1], Z [m], Hbar [(m+1) x m])
    before any rotation, for checking the relation A Z_m = V_{m+1} Hbar_m."""
    beta = np.linalg.norm(r0)
    V = [r0 / beta]
    Z = []
    H = np.zeros((m + 1, m), dtype=np.complex128)
    for j in range(m):
        z = M(V[j])
        Z.append(z)
        w = A(z)
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        V.append(w / H[j + 1, j])
    return V, Z, H
