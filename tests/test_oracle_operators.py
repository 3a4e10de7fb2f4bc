"""Pins of the oracle's operator, transfer and multigrid code against facts the
paper and the mathematics fix (no GPU)."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import helmholtz as hz
from oracle import multigrid as mg

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_golden_constants_used_by_oracle():
    # Eq. (8) kernels and the SL shift as the oracle uses them
    assert np.allclose(mg.R_KERNEL, np.array(GOLD["restriction_kernel"]["value"]) * GOLD["restriction_kernel"]["scale"])
    assert np.allclose(mg.P_KERNEL, np.array(GOLD["prolongation_kernel"]["value"]) * GOLD["prolongation_kernel"]["scale"])
    assert np.isclose(hz.omega_h_for_ppw(1.0), GOLD["ppw_rule"]["value"])
    k2 = np.full((2, 2), 0.7)
    m = hz.sl_mass(k2, 0.5)
    assert np.allclose(m, 0.25 * 0.7 * (GOLD["sl_alpha"]["value"] - 1j * GOLD["sl_beta"]["value"]))


def test_stencil_dst_eigenvalues():
    """Constant kappa, constant gamma, no layer: the 5-point operator is diagonalised
    by DST-I; eigenvalue (4 - 2cos(pi k/(N+1)) - 2cos(pi l/(N+1))) - (wh)^2 k^2 (1 - g i)."""
    N = 24
    kappa = np.full((N, N), 0.8)
    p = hz.Problem(kappa, 0, omega_h=0.6, gamma0=0.03)
    i = np.arange(1, N + 1)
    for (k, l) in [(1, 1), (3, 7), (24, 2), (12, 12)]:
        mode = np.outer(np.sin(np.pi * k * i / (N + 1)), np.sin(np.pi * l * i / (N + 1)))
        lam = 4 - 2 * np.cos(np.pi * k / (N + 1)) - 2 * np.cos(np.pi * l / (N + 1)) - 0.36 * 0.64 * (1 - 0.03j)
        assert np.allclose(p.A(mode), lam * mode, atol=1e-13)


def test_stencil_matches_loops_and_is_complex_symmetric():
    N = 10
    kappa = synth.grf_kappa(6, 2, 2.0, 3)
    p = hz.Problem(kappa, 2)
    x = synth.random_complex((N, N), 4)
    assert np.allclose(p.A(x), hz.apply_stencil_loops(p.mass_A, x), atol=1e-14)
    A = mg.dense_matrix(p.mass_A)
    assert np.allclose(A, A.T)                      # complex symmetric, not Hermitian
    assert not np.allclose(A, A.conj().T)
    # a unit vector at an interior node: 4 - m on the diagonal, -1 at the 4 neighbours
    e = np.zeros((N, N), complex)
    e[4, 5] = 1
    col = p.A(e)
    assert np.isclose(col[4, 5], 4 - p.mass_A[4, 5])
    for (a, b) in [(3, 5), (5, 5), (4, 4), (4, 6)]:
        assert col[a, b] == -1
    assert np.count_nonzero(col) == 5


def test_abl_profile_and_frequency_rule():
    N, L = 40, 8
    g = hz.abl_gamma(N, L)
    assert g[N // 2, N // 2] == 0 and g[L, L] == 0 and g[N - 1 - L, N // 2] == 0
    assert g[0, N // 2] == 1 and g[N - 1, N // 2] == 1 and g[0, 0] == 1
    assert np.isclose(g[L - 4, N // 2], 0.25)      # quadratic ramp, half-way in
    kappa = synth.grf_kappa(N - 2 * L, L, 4.0, 1)
    assert np.isclose(kappa.max(), 1.0) and np.isclose(kappa.min(), 0.25)
    p = hz.Problem(kappa, L)
    assert np.isclose(p.omega_h * kappa.max(), 2 * np.pi / 10)


def _mat(f, n_in):
    I = np.eye(n_in * n_in).reshape(n_in * n_in, n_in, n_in)
    return np.stack([f(v).ravel() for v in I], axis=1)


def test_restriction_is_quarter_prolongation_transpose():
    R = _mat(mg.restrict, 12)
    P = _mat(mg.prolong, 6)
    assert np.array_equal(R, P.T / 4)


def test_prolongation_exact_on_bilinear_and_restriction_on_constants():
    n = 8
    J = np.arange(n)
    # coarse samples of a bilinear function at fine coordinates 2J
    f = lambda y, x: 1.5 + 0.25 * y - 0.5 * x + 0.125 * x * y
    ec = f(2.0 * J[:, None], 2.0 * J[None, :])
    fine = mg.prolong(ec)
    y = np.arange(2 * n)
    exact = f(y[:, None].astype(float), y[None, :].astype(float))
    # exact wherever both coarse neighbours exist (all fine points except the last row/col)
    assert np.allclose(fine[:-1, :-1], exact[:-1, :-1])
    c = np.full((16, 16), 3.0)
    rc = mg.restrict(c)
    assert np.allclose(rc[1:, 1:], 3.0)          # interior: weights sum to 1
    assert np.isclose(rc[0, 0], 3.0 * 9 / 16)    # corner loses the out-of-grid weights
    assert np.allclose(mg.restrict_average(c), 3.0)


def _vcycle_error_radius(N, levels, nu):
    p0 = hz.Problem(np.ones((N, N)), 0, omega_h=0.0)
    M = mg.SLMultigrid(p0, levels, nu1=nu, nu2=nu, coarse="lu")
    A = mg.dense_matrix(np.zeros((N, N)))
    I = np.eye(N * N).reshape(N * N, N, N).astype(complex)
    BV = np.stack([M(v).ravel() for v in I], axis=1)
    return np.abs(np.linalg.eigvals(np.eye(N * N) - BV @ A)).max(), BV


@pytest.mark.parametrize("levels", [2, 3])
def test_vcycle_factor_at_omega_zero_matches_lfa(levels):
    """At omega = 0 the SL operator is -Delta_h.  Local Fourier analysis of damped
    Jacobi (w = 0.8) gives the smoothing factor mu = max(|1-2w|, |1-w/2|) = 0.6, so
    V(1,1) ~ mu^2 = 0.36 and V(2,2) ~ mu^4 = 0.13 (so the paper's 0.2 is read as a V(2,2) bound)."""
    rho1, BV = _vcycle_error_radius(32, levels, 1)
    rho2, _ = _vcycle_error_radius(32, levels, 2)
    assert 0.30 < rho1 <= 0.40
    assert rho2 < 0.2
    # with an exact coarse solve the cycle is a complex-symmetric linear operator
    assert np.allclose(BV, BV.T, atol=1e-12)


def test_two_grid_equals_explicit_matrix_formula():
    N = 16
    kappa = synth.grf_kappa(12, 2, 3.0, 5)
    p = hz.Problem(kappa, 2)
    M = mg.SLMultigrid(p, 2, coarse="lu")
    S0 = mg.dense_matrix(M.mass[0])
    Sc = mg.dense_matrix(M.mass[1])
    R = _mat(mg.restrict, N)
    P = _mat(mg.prolong, N // 2)
    Dinv = np.diag(1.0 / np.diag(S0))
    # Algorithm 1 as matrices: pre-smooth from zero, coarse correction with the
    # h^2-scaled residual 4 R (r - S0 u), post-smooth
    pre = 0.8 * Dinv
    B = pre + P @ np.linalg.solve(Sc, 4 * R @ (np.eye(N * N) - S0 @ pre))
    B = B + 0.8 * Dinv @ (np.eye(N * N) - S0 @ B)
    r = synth.random_complex((N, N), 9)
    assert np.allclose(M(r).ravel(), B @ r.ravel(), atol=1e-12)


def test_coarse_gmres_jacobi_converges_to_lu():
    N = 12
    kappa = synth.grf_kappa(N, 0, 3.0, 2)
    p = hz.Problem(kappa, 0)
    mass = hz.sl_mass(kappa ** 2, p.omega_h * 4)
    r = synth.random_complex((N, N), 3)
    x_lu = np.linalg.solve(mg.dense_matrix(mass), r.ravel()).reshape(N, N)
    x10 = mg.gmres_jacobi_fixed(mass, r, 10)
    xfull = mg.gmres_jacobi_fixed(mass, r, N * N)
    assert np.linalg.norm(xfull - x_lu) < 1e-8 * np.linalg.norm(x_lu)
    # 10 iterations reduce the residual (minimal residual property over D^-1 K_10)
    res10 = np.linalg.norm(r - hz.apply_stencil(mass, x10))
    res5 = np.linalg.norm(r - hz.apply_stencil(mass, mg.gmres_jacobi_fixed(mass, r, 5)))
    assert res10 < res5 < np.linalg.norm(r)


def test_rectangular_grids_reduce_to_the_square_definitions():
    """Rectangular grids (square cells): each axis of gamma is the square profile of its
    own length, the stencil equals the element-by-element brute force, and FGMRES with
    the V-cycle solves the assembled system (dense LU) on a small rectangular grid."""
    from oracle import fgmres as ofg
    N, M, L = 24, 40, 4
    g = hz.abl_gamma(N, L, 0.0, M)
    assert g.shape == (N, M)
    assert np.array_equal(g[N // 2], hz.abl_gamma(M, L)[M // 2])      # row through the middle
    assert np.array_equal(g[:, M // 2], hz.abl_gamma(N, L)[:, N // 2])
    rng = np.random.default_rng(4)
    kappa = 0.25 + 0.75 * rng.random((N, M))
    p = hz.Problem(kappa, L)
    x = rng.standard_normal((N, M)) + 1j * rng.standard_normal((N, M))
    assert np.allclose(p.A(x), hz.apply_stencil_loops(p.mass_A, x), atol=1e-13)
    b = rng.standard_normal((N, M)) + 1j * rng.standard_normal((N, M))
    mgp = mg.SLMultigrid(p, 3, coarse="lu")
    xs, res = ofg.fgmres(p.A, b, np.zeros_like(b), mgp, 20, 1e-12, 400)
    ref = np.linalg.solve(mg.dense_matrix(p.mass_A), b.ravel()).reshape(N, M)
    assert np.linalg.norm(xs - ref) <= 1e-9 * np.linalg.norm(ref)
