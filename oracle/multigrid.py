"""Oracle: shifted-Laplacian geometric multigrid (Section 3.2, Eq. 4, 6, 8, Algorithm 1;
coarsest solve per Section 3.4).

Test infrastructure only (see the package docstring).

Conventions (readings of the paper where it is silent):
  * Grid: unknowns at 0..N-1 with zero values at -1 and N.  Coarse point J sits
    at fine point 2J; N must be even at every level that is coarsened.
  * Restriction I_h^H (Eq. 8): stride-2 correlation with (1/16)[1 2 1;2 4 2;1 2 1],
    zero padding, output N/2.  Prolongation I_H^h (Eq. 8): stride-2 transposed
    correlation with (1/4)[1 2 1;2 4 2;1 2 1], output 2N.  Hence R = P^T / 4.
  * Operators are h_l^2-scaled at every level, so the coarse right-hand side of
    Eq. (6) becomes 4 * R(residual) (H^2 = 4 h^2).
  * Coarse operators are rediscretised (same 5-point stencil at h_l = 2^l h) with
    kappa^2 restricted by full weighting, normalised by the weight that falls
    inside the grid.
  * Boundary of the coarse grids: with N even and coarse point J at fine 2J, the
    high-side Dirichlet boundary of every level coincides with the fine one, but
    on the low side (index -1) the fine boundary lies h = H_l / 2^l before the
    first coarse row/column instead of H_l.  The rediscretised operator keeps the
    boundary where the fine grid has it: the ghost value from linear
    extrapolation through that zero is -(2^l - 1) u_0, which adds 2^l - 1 to the
    diagonal of the first row and column (folded into the mass term).  Without it
    the 3-level cycle diverges at omega = 0 (spectral radius 1.18 on 32^2).
  * Neumann and Sommerfeld problems (see oracle.helmholtz): every level is
    rediscretised with the same boundary condition, c times the boundary sides added
    to its mass with kappa_l = sqrt(restricted kappa^2) and h_l = 2^l h; the low-side
    correction above belongs to the Dirichlet condition only.
  * Relaxation: damped Jacobi u <- u + w D^{-1} (r - M u), D = diag(M), w = 0.8,
    one pre- and one post-sweep (Section 3.4), zero initial guess on every level.
  * Coarsest level: either a dense LU solve, or a fixed number (10) of GMRES
    iterations with Jacobi right-preconditioning from a zero guess (Section 3.4),
    always run to the full count so the map is deterministic.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .helmholtz import apply_stencil, boundary_mass, sl_mass

FW = np.array([[1.0, 2.0, 1.0], [2.0, 4.0, 2.0], [1.0, 2.0, 1.0]])
R_KERNEL = FW / 16.0   # I_h^H, Eq. (8)
P_KERNEL = FW / 4.0    # I_H^h, Eq. (8)


def restrict(x: np.ndarray) -> np.ndarray:
    """Full-weighting restriction I_h^H (Eq. 8): y[J,K] = sum_{a,b} R[a,b] x[2J+a, 2K+b],
    a, b in {-1,0,1}, zero outside the fine grid.  [..., N, M] -> [..., N/2, M/2]."""
    N, M = x.shape[-2:]
    assert N % 2 == 0 and M % 2 == 0
    xp = np.zeros(x.shape[:-2] + (N + 2, M + 2), dtype=x.dtype)
    xp[..., 1:-1, 1:-1] = x
    y = np.zeros(x.shape[:-2] + (N // 2, M // 2), dtype=x.dtype)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            y += R_KERNEL[a + 1, b + 1] * xp[..., 1 + a:1 + a + N:2, 1 + b:1 + b + M:2]
    return y


def prolong(e: np.ndarray) -> np.ndarray:
    """Bilinear prolongation I_H^h (Eq. 8) as a stride-2 transposed correlation:
    fine[2J+a, 2K+b] += P[a,b] e[J,K], a, b in {-1,0,1}; output [..., 2n, 2m]
    (the contribution that would land at fine index -1 falls outside and is dropped)."""
    n, m = e.shape[-2:]
    full = np.zeros(e.shape[:-2] + (2 * n + 2, 2 * m + 2), dtype=e.dtype)  # fine index f -> f+1
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            full[..., 1 + a:1 + a + 2 * n:2, 1 + b:1 + b + 2 * m:2] += P_KERNEL[a + 1, b + 1] * e
    return full[..., 1:1 + 2 * n, 1:1 + 2 * m]


def restrict_average(f: np.ndarray) -> np.ndarray:
    """Full-weighting average of a coefficient field: restrict(f) / restrict(1),
    so coarse values near the boundary are weighted means of in-grid values."""
    return restrict(f) / restrict(np.ones_like(f))


def dense_matrix(mass: np.ndarray) -> np.ndarray:
    """Assemble the h^2-scaled 5-point operator with pointwise `mass` as a dense
    matrix by applying it to every unit vector (row-major unknown ordering)."""
    n, m = mass.shape
    I = np.eye(n * m, dtype=np.complex128).reshape(n * m, n, m)
    return apply_stencil(mass, I).reshape(n * m, n * m).T


def gmres_jacobi_fixed(mass: np.ndarray, r: np.ndarray, iters: int) -> np.ndarray:
    """Coarsest-grid solver of Section 3.4: `iters` GMRES iterations on S e = r with
    right preconditioner D^{-1} (Jacobi), zero initial guess, modified Gram-Schmidt
    Arnoldi, least-squares solution of the small Hessenberg system.  Runs the full
    count unless the Krylov space becomes invariant (h_{j+1,j} == 0)."""
    dinv = 1.0 / (4.0 - mass)
    beta = np.linalg.norm(r)
    if beta == 0.0:
        return np.zeros_like(r)
    V = [r / beta]
    H = np.zeros((iters + 1, iters), dtype=np.complex128)
    k = iters
    for j in range(iters):
        w = apply_stencil(mass, dinv * V[j])
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] == 0.0:
            k = j + 1
            break
        V.append(w / H[j + 1, j])
    rhs = np.zeros(k + 1, dtype=np.complex128)
    rhs[0] = beta
    y = np.linalg.lstsq(H[:k + 1, :k], rhs, rcond=None)[0]
    u = np.zeros_like(r)
    for i in range(k):
        u = u + y[i] * V[i]
    return dinv * u


class SLMultigrid:
    """Shifted-Laplacian V-cycle preconditioner  V(r) ~ M_SL^{-1} r.

    problem      : oracle.helmholtz.Problem (supplies kappa, omega*h, gamma)
    levels       : number of grid levels (>= 2)
    beta         : imaginary shift of Eq. (4) (alpha = 1)
    omega_j      : Jacobi damping
    nu1, nu2     : pre- and post-relaxation sweeps (Algorithm 1)
    coarse       : 'gmres' (Section 3.4 default) or 'lu'
    coarse_iters : GMRES iterations on the coarsest level
    sl_includes_gamma : ablation flag, shift (1 - (beta+gamma) i)
    boundary_fix : keep the low-side Dirichlet boundary at the fine position (default;
                   Dirichlet problems only)
    """

    def __init__(self, problem, levels: int, beta: float = 0.5, omega_j: float = 0.8,
                 nu1: int = 1, nu2: int = 1, coarse: str = "gmres", coarse_iters: int = 10,
                 sl_includes_gamma: bool = False, boundary_fix: bool = True):
        self.levels = levels
        self.omega_j = omega_j
        self.nu1, self.nu2 = nu1, nu2
        self.coarse = coarse
        self.coarse_iters = coarse_iters
        k2 = problem.kappa ** 2
        g = problem.gamma
        bc = getattr(problem, "bc", "dirichlet")
        self.mass = []
        for l in range(levels):
            oh = problem.omega_h * (2 ** l)
            m = sl_mass(k2, oh, beta, gamma=g if sl_includes_gamma else None)
            if bc != "dirichlet":
                m = m + boundary_mass(np.sqrt(k2), oh, bc)
            elif boundary_fix and l > 0:
                m = m.copy()
                m[0, :] -= 2 ** l - 1
                m[:, 0] -= 2 ** l - 1
            self.mass.append(m)
            if l < levels - 1:
                assert k2.shape[0] % 2 == 0 and k2.shape[1] % 2 == 0, "grid not divisible"
                k2 = restrict_average(k2)
                g = restrict_average(g)
        if coarse == "lu":
            self.lu = scipy.linalg.lu_factor(dense_matrix(self.mass[-1]))

    def S(self, l: int, u: np.ndarray) -> np.ndarray:
        """h_l^2-scaled shifted Laplacian at level l."""
        return apply_stencil(self.mass[l], u)

    def coarse_solve(self, r: np.ndarray) -> np.ndarray:
        if self.coarse == "lu":
            shp = r.shape
            return scipy.linalg.lu_solve(self.lu, r.reshape(-1)).reshape(shp)
        return gmres_jacobi_fixed(self.mass[-1], r, self.coarse_iters)

    def relax(self, l: int, u: np.ndarray, r: np.ndarray) -> np.ndarray:
        """One damped-Jacobi sweep on S_l u = r."""
        dinv = 1.0 / (4.0 - self.mass[l])
        return u + self.omega_j * dinv * (r - self.S(l, u))

    def vcycle(self, r: np.ndarray, l: int = 0) -> np.ndarray:
        """Algorithm 1 applied recursively, zero initial guess, one RHS [N][N]."""
        if l == self.levels - 1:
            return self.coarse_solve(r)
        u = np.zeros_like(r)
        for _ in range(self.nu1):
            u = self.relax(l, u, r)
        rc = 4.0 * restrict(r - self.S(l, u))        # Eq. (6), h^2 scaling
        ec = self.vcycle(rc, l + 1)
        u = u + prolong(ec)
        for _ in range(self.nu2):
            u = self.relax(l, u, r)
        return u

    def __call__(self, r: np.ndarray) -> np.ndarray:
        if r.ndim == 2:
            return self.vcycle(r)
        return np.stack([self.vcycle(ri) for ri in r])
