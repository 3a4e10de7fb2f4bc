"""Oracle: the discrete heterogeneous Helmholtz operator (Section 3.1, Eq. 1-3).

Test infrastructure only (see the package docstring).

All operators here act on the h^2-scaled system h^2 A u = h^2 g, so the stencil
entries are O(1):

    (h^2 A u)[i,j] = 4 u[i,j] - u[i-1,j] - u[i+1,j] - u[i,j-1] - u[i,j+1]
                     - (omega h)^2 kappa[i,j]^2 (1 - gamma[i,j] i) u[i,j]

with zero values outside 0..N-1 (zero padding = Dirichlet, Section 3.4).  Eq. (3)
omits gamma "for simplicity"; Eq. (1) carries it, so the mass term here does.

Other boundary conditions (Section 3.4 remark: Neumann by replication padding; Section
3.1: Sommerfeld as an alternative to the absorbing layer) replace the zero ghost values
by multiples of the boundary value, u_ghost = c u_b, so each boundary side of a node
adds c to its mass term (the diagonal 4 loses c) and the stencil itself is unchanged:
    dirichlet   c = 0
    neumann     c = 1                  (replication: u_ghost = u_b)
    sommerfeld  c = 1 - i omega h kappa_b
The Sommerfeld value is the first-order one-sided discretisation of the outgoing-wave
condition du/dn + i omega kappa u = 0; with the paper's damping sign (1 - gamma i),
outgoing waves behave as exp(-i k r).
"""
from __future__ import annotations

import numpy as np


def omega_h_for_ppw(kappa_max: float = 1.0, ppw: float = 10.0) -> float:
    """omega*h from the points-per-wavelength rule omega*kappa*h <= 2*pi/ppw
    (Section 3.1, after Eq. 3), taken with equality at the largest kappa
    (shortest wavelength)."""
    return 2.0 * np.pi / (ppw * kappa_max)


def _abl_profile(N: int, abl: int) -> np.ndarray:
    i = np.arange(N)
    d = np.maximum(np.maximum(abl - i, i - (N - 1 - abl)), 0).astype(np.float64)
    return (d / abl) ** 2 if abl > 0 else np.zeros(N)


def abl_gamma(N: int, abl: int, gamma0: float = 0.0, M: int | None = None) -> np.ndarray:
    """Attenuation field gamma(x) = gamma0 + gamma_ABL(x) on an N x M grid (rows x
    columns; M = N by default).

    Section 3.1: the absorbing boundary layer is a function in gamma that goes
    from 0 to 1 towards the boundaries.  Reading: with d = distance in cells into
    the layer (0 at the first interior index `abl`, `abl` at the outermost cell),
    gamma_ABL = max((d_x/L)^2, (d_y/L)^2).
    """
    py = _abl_profile(N, abl)
    px = py if M is None or M == N else _abl_profile(M, abl)
    return gamma0 + np.maximum(py[:, None], px[None, :])


def helmholtz_mass(kappa: np.ndarray, omega_h: float, gamma: np.ndarray) -> np.ndarray:
    """Mass term of h^2 A (Eq. 1 and 3): (omega h)^2 kappa^2 (1 - gamma i)."""
    return (omega_h ** 2) * kappa.astype(np.float64) ** 2 * (1.0 - 1j * gamma)


def sl_mass(kappa2: np.ndarray, omega_h: float, beta: float = 0.5, alpha: float = 1.0,
            gamma: np.ndarray | None = None) -> np.ndarray:
    """Mass term of the h^2-scaled shifted Laplacian (Eq. 4):
    (omega h)^2 kappa^2 (alpha - beta i), alpha = 1, beta = 0.5 (Section 3.2).
    If `gamma` is given (ablation flag), the shift becomes (alpha - (beta+gamma) i).
    """
    shift = alpha - 1j * (beta + (gamma if gamma is not None else 0.0))
    return (omega_h ** 2) * kappa2 * shift


BOUNDARY_CONDITIONS = ("dirichlet", "neumann", "sommerfeld")


def boundary_sides(N: int, M: int) -> np.ndarray:
    """Number of grid sides a node lies on (0 inside, 1 on an edge, 2 at a corner)."""
    i = np.arange(N)[:, None]
    j = np.arange(M)[None, :]
    return (i == 0).astype(np.float64) + (i == N - 1) + (j == 0) + (j == M - 1)


def ghost_factor(bc: str, kappa: np.ndarray, omega_h: float) -> np.ndarray | float:
    """c in u_ghost = c u_b for the boundary condition `bc` (see the module docstring)."""
    if bc == "dirichlet":
        return 0.0
    if bc == "neumann":
        return 1.0
    if bc == "sommerfeld":
        return 1.0 - 1j * omega_h * np.asarray(kappa, dtype=np.float64)
    raise ValueError(bc)


def boundary_mass(kappa: np.ndarray, omega_h: float, bc: str) -> np.ndarray:
    """The boundary condition folded into the mass term: c times the number of
    boundary sides of each node (zero for Dirichlet)."""
    N, M = np.shape(kappa)
    return boundary_sides(N, M) * ghost_factor(bc, kappa, omega_h) + 0j


def apply_stencil_ghost(mass: np.ndarray, x: np.ndarray, bc: str, kappa: np.ndarray, omega_h: float) -> np.ndarray:
    """The definition of a boundary condition: pad one [N, M] grid with ghost values
    u_ghost = c u_b and apply the 5-point stencil (mass without the boundary term)."""
    N, M = x.shape
    c = np.broadcast_to(ghost_factor(bc, kappa, omega_h), (N, M))
    xp = np.zeros((N + 2, M + 2), dtype=np.complex128)
    xp[1:-1, 1:-1] = x
    xp[0, 1:-1] = c[0, :] * x[0, :]
    xp[-1, 1:-1] = c[-1, :] * x[-1, :]
    xp[1:-1, 0] = c[:, 0] * x[:, 0]
    xp[1:-1, -1] = c[:, -1] * x[:, -1]
    nbr = xp[:-2, 1:-1] + xp[2:, 1:-1] + xp[1:-1, :-2] + xp[1:-1, 2:]
    return (4.0 - mass) * x - nbr


def apply_stencil(mass: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = (h^2 A) x for the 5-point operator of Eq. (3) with a pointwise mass.

    `x` is [..., N, M] (any leading batch dims); `mass` is [N, M].  Zero padding
    outside the grid (Section 3.4: zero-padded convolutions = Dirichlet BC).
    """
    x = np.asarray(x)
    xp = np.zeros(x.shape[:-2] + (x.shape[-2] + 2, x.shape[-1] + 2), dtype=np.result_type(x, mass))
    xp[..., 1:-1, 1:-1] = x
    nbr = xp[..., :-2, 1:-1] + xp[..., 2:, 1:-1] + xp[..., 1:-1, :-2] + xp[..., 1:-1, 2:]
    return (4.0 - mass) * x - nbr


def apply_stencil_loops(mass: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Element-by-element version of `apply_stencil` for tiny grids (brute force)."""
    N, M = x.shape
    y = np.zeros((N, M), dtype=np.complex128)
    for i in range(N):
        for j in range(M):
            s = (4.0 - mass[i, j]) * x[i, j]
            for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < N and 0 <= jj < M:
                    s -= x[ii, jj]
            y[i, j] = s
    return y


class Problem:
    """One slowness model with its frequency and absorbing layer.

    kappa   : float64 [ny][nx] slowness (including the absorbing layer cells); square
              (the paper's setting) or rectangular with square cells
    abl     : layer width in cells
    omega_h : omega * h (dimensionless); default from the 10 points-per-wavelength rule
    gamma0  : constant attenuation (0 at solve time, 0.05 when generating training
              data, Section 4.3)
    bc      : boundary condition outside the grid: 'dirichlet' (zero padding, the
              paper's setting), 'neumann' or 'sommerfeld' (folded into the mass term)
    """

    def __init__(self, kappa: np.ndarray, abl: int, omega_h: float | None = None,
                 gamma0: float = 0.0, bc: str = "dirichlet"):
        self.kappa = np.asarray(kappa, dtype=np.float64)
        assert self.kappa.ndim == 2
        self.N, self.M = self.kappa.shape
        self.abl = abl
        self.bc = bc
        self.omega_h = omega_h_for_ppw(self.kappa.max()) if omega_h is None else omega_h
        self.gamma = abl_gamma(self.N, abl, gamma0, self.M)
        self.mass_A = helmholtz_mass(self.kappa, self.omega_h, self.gamma)
        if bc != "dirichlet":
            self.mass_A = self.mass_A + boundary_mass(self.kappa, self.omega_h, bc)

    def A(self, x: np.ndarray) -> np.ndarray:
        """h^2 A x (Eq. 3 with gamma)."""
        return apply_stencil(self.mass_A, x)
