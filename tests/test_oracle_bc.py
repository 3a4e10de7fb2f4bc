"""Pins of the oracle's boundary conditions other than Dirichlet (Section 3.4: Neumann by
replication padding; Section 3.1: Sommerfeld as an alternative to the absorbing layer)
against their definitions and against the mathematics (no GPU)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl
from scipy.special import hankel2

import synth
from oracle import fgmres as ofg
from oracle import helmholtz as hz
from oracle import multigrid as mg


def _sparse(mass):
    """The zero-padded 5-point operator (4 - mass) u - sum of neighbours, assembled
    with scipy.sparse as a Kronecker sum (rows i, columns j, row-major)."""
    N, M = mass.shape

    def second_difference(n):
        return sp.diags([-np.ones(n - 1), np.zeros(n), -np.ones(n - 1)], [-1, 0, 1])

    A = sp.kron(sp.eye(N), second_difference(M)) + sp.kron(second_difference(N), sp.eye(M))
    return (A + sp.diags((4.0 - mass).ravel())).tocsc()


@pytest.mark.parametrize("bc", hz.BOUNDARY_CONDITIONS)
def test_boundary_condition_folds_into_the_mass_term(bc):
    """The folded operator equals the ghost-value definition: u_ghost = u_b
    (replication, Neumann), (1 - i omega h kappa_b) u_b (first-order Sommerfeld),
    0 (Dirichlet), on a rectangular grid with an absorbing layer and random kappa."""
    rng = np.random.default_rng(7)
    N, M, L = 12, 20, 3
    kappa = 0.25 + 0.75 * rng.random((N, M))
    p = hz.Problem(kappa, L, bc=bc)
    plain = hz.helmholtz_mass(p.kappa, p.omega_h, p.gamma)
    for _ in range(3):
        x = rng.standard_normal((N, M)) + 1j * rng.standard_normal((N, M))
        ref = hz.apply_stencil_ghost(plain, x, bc, p.kappa, p.omega_h)
        assert np.allclose(p.A(x), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    # the boundary terms sit on the outermost ring only, twice at the corners
    extra = p.mass_A - plain
    assert np.all(extra[1:-1, 1:-1] == 0)
    if bc != "dirichlet":
        assert np.isclose(extra[0, 0], 2 * hz.ghost_factor(bc, kappa[0, 0], p.omega_h))
        assert np.isclose(extra[0, 5], hz.ghost_factor(bc, kappa[0, 5], p.omega_h))
    # complex symmetric in every case (the ghost values only change the diagonal)
    D = mg.dense_matrix(p.mass_A)
    assert np.allclose(D, D.T, atol=0)


def test_neumann_eigenpairs_are_the_dct():
    """Replication padding makes the 1D second difference the cell-centred Neumann one,
    diagonalised by the DCT-II: for constant kappa and gamma (no layer), A v = lambda v
    with v = cos(pi k (i + 1/2)/N) cos(pi l (j + 1/2)/M) and
    lambda = 4 - 2 cos(pi k/N) - 2 cos(pi l/M) - (omega h)^2 kappa^2 (1 - gamma i)."""
    N, M = 10, 14
    kappa = np.full((N, M), 0.7)
    p = hz.Problem(kappa, 0, omega_h=0.4, gamma0=0.02, bc="neumann")
    i = np.arange(N)[:, None]
    j = np.arange(M)[None, :]
    m = 0.4 ** 2 * 0.49 * (1 - 0.02j)
    for k, l in ((0, 0), (1, 0), (0, 3), (4, 7), (N - 1, M - 1)):
        v = np.cos(np.pi * k * (i + 0.5) / N) * np.cos(np.pi * l * (j + 0.5) / M)
        lam = 4 - 2 * np.cos(np.pi * k / N) - 2 * np.cos(np.pi * l / M) - m
        assert np.allclose(p.A(v), lam * v, atol=1e-12)
    # at omega = 0 the Neumann Laplacian annihilates constants; the Dirichlet one does not
    one = np.ones((N, M))
    assert np.abs(hz.Problem(kappa, 0, omega_h=0.0, bc="neumann").A(one)).max() < 1e-14
    assert np.abs(hz.Problem(kappa, 0, omega_h=0.0).A(one)).max() >= 1.0


def test_sommerfeld_absorbs_on_the_boundary():
    """For real kappa the imaginary part of x^H A x is the attenuation inside plus the
    boundary absorption: sum (omega h)^2 kappa^2 gamma |x|^2 + omega h sum n_b kappa |x|^2,
    n_b the number of boundary sides of a node (positive for every x != 0)."""
    rng = np.random.default_rng(2)
    N, M, L = 16, 12, 3
    kappa = 0.25 + 0.75 * rng.random((N, M))
    p = hz.Problem(kappa, L, bc="sommerfeld")
    nb = hz.boundary_sides(N, M)
    for _ in range(3):
        x = rng.standard_normal((N, M)) + 1j * rng.standard_normal((N, M))
        q = np.vdot(x, p.A(x))
        ref = (p.omega_h ** 2 * kappa ** 2 * p.gamma * np.abs(x) ** 2).sum() \
            + p.omega_h * (nb * kappa * np.abs(x) ** 2).sum()
        assert np.isclose(q.imag, ref, rtol=1e-12)
    # the Neumann operator has no boundary term in its imaginary part
    pn = hz.Problem(kappa, L, bc="neumann")
    x = rng.standard_normal((N, M)) + 1j * rng.standard_normal((N, M))
    ref = (pn.omega_h ** 2 * kappa ** 2 * pn.gamma * np.abs(x) ** 2).sum()
    assert np.isclose(np.vdot(x, pn.A(x)).imag, ref, rtol=1e-12)


def test_sommerfeld_point_source_approaches_the_free_space_green_function():
    """Unit point source, constant kappa, no layer and no attenuation, 20 points per
    wavelength: with the outgoing-wave condition the discrete solution is close to the
    free-space Green's function (-i/4) H0^(2)(k r) of -Delta - k^2 (outgoing waves are
    exp(-i k r) under the paper's damping sign).  The residual difference is dispersion
    and the first-order condition's oblique reflection.  Walls (Dirichlet, Neumann) and
    the condition with the wrong sign are far from it."""
    N = 129
    oh = 2 * np.pi / 20
    kappa = np.ones((N, N))
    c = N // 2
    b = np.zeros(N * N, dtype=np.complex128)
    b[c * N + c] = 1.0                      # h^2 g with g = delta / h^2
    i = np.arange(N)[:, None]
    j = np.arange(N)[None, :]
    kr = np.hypot(i - c, j - c) * oh
    G = -0.25j * hankel2(0, np.where(kr > 0, kr, 1.0))
    ring = (kr > 3 * 2 * np.pi / 10) & (np.hypot(i - c, j - c) < 0.4 * N)
    x = np.random.default_rng(0).standard_normal((N, N)) + 0j

    def err(mass):
        A = _sparse(mass)
        assert np.allclose(A @ x.ravel(), hz.apply_stencil(mass, x).ravel(), atol=1e-13)
        u = spl.spsolve(A, b).reshape(N, N)
        return np.linalg.norm((u - G)[ring]) / np.linalg.norm(G[ring])

    e = {bc: err(hz.Problem(kappa, 0, omega_h=oh, bc=bc).mass_A) for bc in hz.BOUNDARY_CONDITIONS}
    # the condition with the sign flipped: ghost = (1 + i omega h kappa) u_b
    wrong = hz.helmholtz_mass(kappa, oh, np.zeros((N, N))) + hz.boundary_sides(N, N) * (1 + 1j * oh)
    e["wrong sign"] = err(wrong)
    assert e["sommerfeld"] < 0.15, e
    assert min(e["dirichlet"], e["neumann"], e["wrong sign"]) > 1.0, e


@pytest.mark.parametrize("bc,abl", [("neumann", 4), ("sommerfeld", 4), ("sommerfeld", 0)])
def test_vcycle_and_fgmres_with_the_boundary_condition(bc, abl):
    """Every multigrid level carries the same condition (kappa_l = sqrt of the restricted
    kappa^2, h_l = 2^l h).  Pinned as for Dirichlet: the two-grid cycle equals its matrix
    formula, the cycle with an exact coarse solve is complex symmetric, and FGMRES with
    the V-cycle solves the system assembled from the ghost-value definition (dense LU)."""
    N = 32
    kappa = synth.grf_kappa(N - 2 * abl, abl, 4.0, 5)
    p = hz.Problem(kappa, abl, bc=bc)
    plain = hz.helmholtz_mass(p.kappa, p.omega_h, p.gamma)
    n = N * N
    E = np.eye(n).reshape(n, N, N)
    Adef = np.stack([hz.apply_stencil_ghost(plain, e, bc, p.kappa, p.omega_h).ravel() for e in E], axis=1)
    # coarse levels: the boundary term of each level
    M3 = mg.SLMultigrid(p, 3, coarse="lu")
    k2c = mg.restrict_average(p.kappa ** 2)
    sl1 = hz.sl_mass(k2c, 2 * p.omega_h)
    assert np.allclose(M3.mass[1], sl1 + hz.boundary_mass(np.sqrt(k2c), 2 * p.omega_h, bc), atol=1e-15)
    # two-grid cycle vs Algorithm 1 written as matrices
    M2 = mg.SLMultigrid(p, 2, coarse="lu")
    S0 = mg.dense_matrix(M2.mass[0])
    Sc = mg.dense_matrix(M2.mass[1])
    R = np.stack([mg.restrict(e).ravel() for e in E], axis=1)
    P = np.stack([mg.prolong(e).ravel() for e in np.eye(n // 4).reshape(n // 4, N // 2, N // 2)], axis=1)
    pre = 0.8 * np.diag(1.0 / np.diag(S0))
    B = pre + P @ np.linalg.solve(Sc, 4 * R @ (np.eye(n) - S0 @ pre))
    B = B + pre @ (np.eye(n) - S0 @ B)
    BV = np.stack([M2(e).ravel() for e in E], axis=1)
    assert np.allclose(BV, B, atol=1e-12)
    assert np.allclose(BV, BV.T, atol=1e-12)
    b = synth.random_complex((N, N), 4)
    xs, res = ofg.fgmres(p.A, b, np.zeros_like(b), mg.SLMultigrid(p, 3), 10, 1e-12, 600)
    ref = np.linalg.solve(Adef, b.ravel()).reshape(N, N)
    assert res.converged and np.linalg.norm(xs - ref) <= 1e-8 * np.linalg.norm(ref)


@pytest.mark.parametrize("bc", ["neumann", "sommerfeld"])
def test_coarse_levels_are_the_same_boundary_value_problem(bc):
    """Every multigrid level carries the condition of the fine problem on its own grid
    (spacing 2^l h, kappa_l = sqrt of the restricted kappa^2).  On levels 0-2 the level's
    operator equals the ghost-value definition of the condition (u_ghost = c_l u_b, c_l
    from kappa_l and omega h_l) applied to the level's shifted-Laplacian mass; and with
    constant kappa it meets the closed forms of the condition on the constant vector:
    the stencil part vanishes for Neumann (S_l 1 = -mass), and each boundary side adds
    i omega h_l kappa for first-order Sommerfeld."""
    N, abl, levels = 32, 4, 3
    rng = np.random.default_rng(11)
    p = hz.Problem(synth.grf_kappa(N - 2 * abl, abl, 4.0, 9), abl, bc=bc)
    M = mg.SLMultigrid(p, levels)
    k2 = p.kappa ** 2
    for l in range(levels):
        oh = p.omega_h * 2 ** l
        if l:
            k2 = mg.restrict_average(k2)
        slm = hz.sl_mass(k2, oh)
        for _ in range(2):
            u = rng.standard_normal(k2.shape) + 1j * rng.standard_normal(k2.shape)
            ref = hz.apply_stencil_ghost(slm, u, bc, np.sqrt(k2), oh)
            assert np.allclose(M.S(l, u), ref, rtol=0, atol=1e-13 * np.abs(ref).max()), l
    kc = 0.6
    pc = hz.Problem(np.full((N, N), kc), abl, bc=bc)
    Mc = mg.SLMultigrid(pc, levels)
    for l in range(levels):
        n = N >> l
        oh = pc.omega_h * 2 ** l
        slm = hz.sl_mass(np.full((n, n), kc ** 2), oh)
        one = np.ones((n, n), dtype=np.complex128)
        sides = (np.arange(n)[:, None] == 0) * 1.0 + (np.arange(n)[:, None] == n - 1) + \
            (np.arange(n)[None, :] == 0) + (np.arange(n)[None, :] == n - 1)
        want = -slm + (0.0 if bc == "neumann" else 1j * oh * kc * sides)
        assert np.allclose(Mc.S(l, one), want, rtol=0, atol=1e-12), l
