"""Pins of the oracle's FGMRES against dense LU, the Arnoldi relation and a library
GMRES (no GPU)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import helmholtz as hz
from oracle import multigrid as mg
from oracle.fgmres import arnoldi_flexible, fgmres


def _problem(n=20, abl=6, seed=0):
    return hz.Problem(synth.grf_kappa(n, abl, 4.0, seed), abl)


def test_fgmres_solution_matches_dense_lu():
    p = _problem()
    N = p.N
    A = mg.dense_matrix(p.mass_A)
    b = synth.centre_source(N)
    M = mg.SLMultigrid(p, 3, coarse="gmres")
    x, res = fgmres(p.A, b, np.zeros_like(b), M, restart=10, tol=1e-12, maxit=500)
    x_lu = np.linalg.solve(A, b.ravel()).reshape(N, N)
    assert res.converged
    assert np.linalg.norm(x - x_lu) <= 1e-9 * np.linalg.norm(x_lu)


def test_arnoldi_relation_and_orthonormal_basis():
    p = _problem(16, 4, 1)
    M = mg.SLMultigrid(p, 2, coarse="gmres")
    r0 = synth.random_complex((p.N, p.N), 2)
    m = 8
    V, Z, H = arnoldi_flexible(p.A, M, r0, m)
    Vm = np.stack([v.ravel() for v in V], axis=1)
    AZ = np.stack([p.A(z).ravel() for z in Z], axis=1)
    assert np.allclose(AZ, Vm @ H, atol=1e-12 * np.abs(AZ).max())
    assert np.allclose(Vm.conj().T @ Vm, np.eye(m + 1), atol=1e-12)


def test_givens_estimate_equals_true_residual():
    p = _problem(16, 4, 3)
    M = mg.SLMultigrid(p, 3, coarse="gmres")
    b = synth.random_complex((p.N, p.N), 4)
    # a single cycle of k steps: the estimate after step k equals ||b - A x_k||
    for k in (3, 7):
        x, res = fgmres(p.A, b, np.zeros_like(b), M, restart=k, tol=0.0, maxit=k)
        true = np.linalg.norm(b - p.A(x)) / np.linalg.norm(b)
        assert abs(res.est_hist[-1] - true) <= 1e-10 * true


def test_identity_preconditioner_matches_library_gmres():
    p = _problem(12, 3, 5)
    N = p.N
    b = synth.random_complex((N, N), 6)
    k = 15
    x, res = fgmres(p.A, b, np.zeros_like(b), lambda v: v, restart=k, tol=0.0, maxit=k)
    op = spla.LinearOperator((N * N, N * N), matvec=lambda v: p.A(v.reshape(N, N)).ravel(),
                             dtype=np.complex128)
    xs, info = spla.gmres(op, b.ravel(), x0=np.zeros(N * N, complex), restart=k, maxiter=1,
                          rtol=1e-30, atol=0.0)
    assert np.allclose(x.ravel(), xs, atol=1e-9 * np.abs(xs).max())


def test_plain_method_small_config_converges():
    """64 x 64 interior + 16-cell layer, GRF kappa (ell = 8), centre source,
    FGMRES(20), tol 1e-6, 3-level V-cycle with an exact (LU) coarsest solve."""
    kappa = synth.grf_kappa(64, 16, 8.0, 0)
    p = hz.Problem(kappa, 16)
    b = synth.centre_source(p.N)
    M = mg.SLMultigrid(p, 3, coarse="lu")
    x, res = fgmres(p.A, b, np.zeros_like(b), M, restart=20, tol=1e-6, maxit=2000)
    assert res.converged
    assert np.linalg.norm(b - p.A(x)) <= 1e-6 * np.linalg.norm(b)
    assert 20 < res.iters < 200
    # the same system with the identity preconditioner needs far more iterations
    _, res0 = fgmres(p.A, b, np.zeros_like(b), lambda v: v, restart=20, tol=1e-6, maxit=res.iters * 3)
    assert not res0.converged
