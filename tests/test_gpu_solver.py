"""GPU parity of the problem setup, stencil, V-cycle and FGMRES kernels against the
FP64 oracle, through the C ABI.

Tolerances (FP32 kernels vs FP64 oracle, unit roundoff u = 2^-24):
  * setup fields: computed in FP64 on the device and rounded once -> |d| <= u |ref|
  * stencil: six rounded operations per output -> |d| <= 8 u (|4-m||x| + sum |x_nb|)
  * V-cycle: a fixed sequence of FP32 stencil sweeps plus 10 coarse GMRES steps;
    rounding is amplified by the coarse GMRES, measured ~1e-6, bound 2e-4 (norm-wise)
  * FGMRES: judged by the true FP64 residual the oracle computes from the GPU x, and
    by the solution error against the oracle's solution at 1e-12.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import fgmres as ofg
from oracle import helmholtz as ohz
from oracle import multigrid as omg

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_17486_gb300 as h
    return h


DEV = "cuda:0"


def _mk(helm, n, abl, levels, seed=0, gamma0=0.0, kind="grf"):
    if kind == "grf":
        kappa = synth.grf_kappa(n, abl, 6.0, seed)
    else:
        kappa = synth.layered_kappa(n, abl, seed=seed)
    kappa32 = kappa.astype(np.float32).astype(np.float64)
    oh = ohz.omega_h_for_ppw(kappa32.max())
    P = helm.Problem(torch.tensor(kappa32, dtype=torch.float32, device=DEV), abl, oh, gamma0=gamma0, levels=levels)
    op = ohz.Problem(kappa32, abl, omega_h=oh, gamma0=gamma0)
    return P, op


def _c64(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.complex64, device=DEV)


def _q(a):
    """Round to complex64 and back (the GPU's view of an input)."""
    return a.astype(np.complex64).astype(np.complex128)


@pytest.mark.parametrize("n,abl,levels", [(48, 8, 3), (256, 16, 4), (80, 8, 4)])
def test_setup_fields_match_oracle(helm, n, abl, levels):
    P, op = _mk(helm, n, abl, levels, seed=1, gamma0=0.01)
    mg = omg.SLMultigrid(op, levels)
    assert np.allclose(P.field("gamma").cpu().numpy(), op.gamma, rtol=U, atol=U)
    mA = P.field("mass_A").cpu().numpy()
    assert np.all(np.abs(mA - op.mass_A) <= 2 * U * np.abs(op.mass_A) + 1e-30)
    for l in range(levels):
        m = P.field("mass_SL", l).cpu().numpy()
        assert np.all(np.abs(m - mg.mass[l]) <= 4 * U * np.abs(mg.mass[l]) + 1e-7), l
        d = P.field("dinv_SL", l).cpu().numpy()
        dref = 0.8 / (4.0 - mg.mass[l])
        assert np.all(np.abs(d - dref) <= 4 * U * np.abs(dref)), l


@pytest.mark.parametrize("n,abl,B", [(48, 8, 3), (112, 8, 1), (512, 32, 2)])
def test_helmholtz_apply_matches_oracle(helm, n, abl, B):
    P, op = _mk(helm, n, abl, 3, seed=2)
    N = op.N
    x = _q(synth.random_complex((B, N, N), 3))
    y = helm.helmholtz_apply(P, _c64(x)).cpu().numpy()
    ref = op.A(x)
    xp = np.pad(np.abs(x), ((0, 0), (1, 1), (1, 1)))
    scale = np.abs(4 - op.mass_A) * np.abs(x) + xp[:, :-2, 1:-1] + xp[:, 2:, 1:-1] + xp[:, 1:-1, :-2] + xp[:, 1:-1, 2:]
    assert np.all(np.abs(y - ref) <= 8 * U * scale)


def test_helmholtz_apply_edges_and_zero(helm):
    P, op = _mk(helm, 48, 8, 3)
    N = op.N
    # unit vectors at the four corners and the edges: zero (Dirichlet) padding
    x = np.zeros((4, N, N), complex)
    for k, (i, j) in enumerate([(0, 0), (N - 1, N - 1), (0, N // 2), (N // 2, N - 1)]):
        x[k, i, j] = 1.0 + 0.5j
    y = helm.helmholtz_apply(P, _c64(x)).cpu().numpy()
    assert np.allclose(y, op.A(x), rtol=4 * U, atol=4 * U)
    z = helm.helmholtz_apply(P, _c64(np.zeros((1, N, N)))).cpu().numpy()
    assert not np.any(z)


def test_residual_fp64_matches_oracle(helm):
    P, op = _mk(helm, 96, 16, 3, seed=4)
    N = op.N
    b = _q(synth.random_complex((2, N, N), 5))
    x = synth.random_complex((2, N, N), 6)
    r, nr = helm.helmholtz_residual_fp64(P, _c64(b), torch.tensor(x, dtype=torch.complex128, device=DEV))
    ref = b - op.A(x)
    # FP64 arithmetic (FP64 mass term), result within one FP32 ulp
    bound = 2 * U * np.abs(ref) + 1e-13 * (np.abs(b) + 10 * np.abs(x))
    assert np.all(np.abs(r.cpu().numpy() - ref) <= bound)
    assert np.allclose(nr.cpu().numpy(), (np.abs(ref) ** 2).sum(axis=(1, 2)), rtol=1e-12)


@pytest.mark.parametrize("n,abl,levels,B", [(48, 8, 3, 2), (64, 16, 4, 3), (256, 16, 4, 2), (40, 4, 2, 1)])
def test_vcycle_matches_oracle(helm, n, abl, levels, B):
    P, op = _mk(helm, n, abl, levels, seed=7)
    N = op.N
    mg = omg.SLMultigrid(op, levels, coarse="gmres", coarse_iters=10)
    r = _q(synth.random_complex((B, N, N), 8))
    z = helm.slmg_vcycle(P, _c64(r)).cpu().numpy()
    for i in range(B):
        zref = mg(r[i])
        err = np.linalg.norm(z[i] - zref) / np.linalg.norm(zref)
        assert err < 2e-4, err
    zero = helm.slmg_vcycle(P, _c64(np.zeros((1, N, N)))).cpu().numpy()
    assert not np.any(zero)


def test_fgmres_matches_oracle_solution(helm):
    """Small problem: GPU FGMRES(10) with the SL V-cycle vs the oracle solved to 1e-12."""
    P, op = _mk(helm, 64, 16, 3, seed=0)
    N = op.N
    b = synth.random_point_sources(N, 16, 3, seed=9)
    b[2] = synth.centre_source(N)
    x, st = helm.fgmres_solve(P, _c64(b), restart=10, rtol=1e-6, maxit=2000)
    xs = x.cpu().numpy()
    mg = omg.SLMultigrid(op, 3)
    for i in range(3):
        assert st["status"][i] == 1
        true = np.linalg.norm(b[i] - op.A(xs[i])) / np.linalg.norm(b[i])
        assert true <= 1e-6 and abs(true - st["rel_res_true"][i]) <= 1e-9
        xr, res = ofg.fgmres(op.A, b[i], np.zeros_like(b[i]), mg, 10, 1e-12, 4000)
        # the residual bounds the error only through ||A^-1||, so the GPU's error at a 1e-6
        # residual is compared with the FP64 oracle's own error at the same residual
        xr6, res6 = ofg.fgmres(op.A, b[i], np.zeros_like(b[i]), mg, 10, 1e-6, 4000)
        rel_err = np.linalg.norm(xs[i] - xr) / np.linalg.norm(xr)
        oracle_err = np.linalg.norm(xr6 - xr) / np.linalg.norm(xr)
        print(f"rhs {i}: solution error GPU {rel_err:.2e}, FP64 oracle at the same tolerance {oracle_err:.2e}")
        assert rel_err < 1e-3, rel_err
        assert rel_err <= 10 * oracle_err + 1e-6, (rel_err, oracle_err)
        assert abs(st["iters"][i] - res6.iters) <= max(3, 0.1 * res6.iters), (st["iters"][i], res6.iters)


def test_fgmres_fixed_iterations_matches_oracle(helm):
    """Data-generation mode (Eq. 17): exactly k iterations from x0 = 0, per-RHS caps."""
    P, op = _mk(helm, 48, 8, 3, seed=2, gamma0=0.05)
    N = op.N
    x_true = synth.smooth_plus_noise(3, N, seed=3)
    b = np.stack([op.A(v) for v in x_true])
    b = _q(b)
    ks = np.array([2, 7, 20], dtype=np.int32)
    caps = torch.tensor(ks, device=DEV)
    xg, st = helm.fgmres_solve(P, _c64(b), restart=20, rtol=0.0, maxit=20, maxit_per_rhs=caps)
    xg = xg.cpu().numpy()
    mg = omg.SLMultigrid(op, 3)
    for i, k in enumerate(ks):
        assert st["iters"][i] == k and st["status"][i] == 2
        xr, _ = ofg.fgmres(op.A, b[i], np.zeros_like(b[i]), mg, int(k), 0.0, int(k))
        err = np.linalg.norm(xg[i] - xr) / np.linalg.norm(xr)
        assert err < 1e-4, (k, err)


def test_fgmres_edge_cases(helm):
    P, op = _mk(helm, 48, 8, 3, seed=5)
    N = op.N
    b = synth.random_point_sources(N, 8, 4, seed=1)
    b[1] = 0.0                               # zero right-hand side -> x = 0, converged
    b[2, 3, 3] = np.nan                      # non-finite input -> NONFINITE, others unaffected
    x0 = np.zeros((4, N, N), complex)
    x0[1] = 1.0
    x, st = helm.fgmres_solve(P, _c64(b), torch.tensor(x0, dtype=torch.complex128, device=DEV), rtol=1e-6)
    xs = x.cpu().numpy()
    assert st["status"][1] == 1 and not np.any(xs[1])
    assert st["status"][2] == 3
    for i in (0, 3):
        assert st["status"][i] == 1
        assert np.linalg.norm(b[i] - op.A(xs[i])) <= 1e-6 * np.linalg.norm(b[i])
    # an exact initial guess converges with zero iterations
    x2, st2 = helm.fgmres_solve(P, _c64(b[:1]), x[:1].clone(), rtol=1e-6)
    assert st2["iters"][0] == 0 and st2["status"][0] == 1
    # maxit reached
    _, st3 = helm.fgmres_solve(P, _c64(b[:1]), rtol=1e-14, maxit=5)
    assert st3["status"][0] == 2 and st3["iters"][0] == 5
    assert helm.device_errors() == 0


@pytest.mark.parametrize("reorth", [0, 1, 2])
def test_fgmres_layered_model_all_orthogonalisations(helm, reorth):
    """256^2 interior + 16-cell layer, layered kappa, 4-level V-cycle (sampled RHS)."""
    P, op = _mk(helm, 256, 16, 4, seed=1, kind="layered")
    N = op.N
    b = synth.random_point_sources(N, 16, 4, seed=21)
    x, st = helm.fgmres_solve(P, _c64(b), restart=10, rtol=1e-6, maxit=2000, reorth=reorth)
    xs = x.cpu().numpy()
    assert np.all(st["status"] == 1), st
    for i in range(4):
        true = np.linalg.norm(b[i] - op.A(xs[i])) / np.linalg.norm(b[i])
        assert true <= 1e-6


def test_full_size_point_sources_true_residual(helm):
    """512^2 interior + 32-cell layer (576^2 grid), GRF kappa, 16 point sources in one
    launch, FGMRES(10) with the 4-level V-cycle: the oracle's FP64 matvec checks every
    returned solution's true residual."""
    P, op = _mk(helm, 512, 32, 4, seed=10)
    N = op.N
    b = synth.random_point_sources(N, 32, 16, seed=10)
    x, st = helm.fgmres_solve(P, _c64(b), restart=10, rtol=1e-6, maxit=3000)
    xs = x.cpu().numpy()
    assert np.all(st["status"] == 1), st
    for i in range(16):
        true = np.linalg.norm(b[i] - op.A(xs[i])) / np.linalg.norm(b[i])
        assert true <= 1e-6
        assert abs(true - st["rel_res_true"][i]) <= 1e-9


def test_rectangular_grid_setup_apply_vcycle_and_solve(helm):
    """A 288 x 160 grid (square cells, 16-cell absorbing layer, 4 levels): setup fields,
    the matvec and one V-cycle element by element against the oracle, and FGMRES judged
    by the oracle's FP64 true residual of the GPU solution."""
    ny, nx, abl, levels, B = 160, 288, 16, 4, 3
    kappa = synth.grf_kappa(nx - 2 * abl, abl, 6.0, 12)[:ny].astype(np.float32).astype(np.float64)
    oh = ohz.omega_h_for_ppw(kappa.max())
    P = helm.Problem(torch.tensor(np.ascontiguousarray(kappa), dtype=torch.float32, device=DEV), abl, oh, levels=levels)
    op = ohz.Problem(kappa, abl, omega_h=oh)
    assert P.level_shape(levels - 1) == (ny >> (levels - 1), nx >> (levels - 1))
    assert np.allclose(P.field("gamma").cpu().numpy(), op.gamma, rtol=U, atol=U)
    x = _q(synth.random_complex((B, ny, nx), 3))
    y = helm.helmholtz_apply(P, _c64(x)).cpu().numpy()
    yref = np.stack([op.A(x[i]) for i in range(B)])
    assert np.abs(y - yref).max() <= 1e-5 * np.abs(yref).max()
    mgp = omg.SLMultigrid(op, levels, coarse="gmres", coarse_iters=10)
    z = helm.slmg_vcycle(P, _c64(x)).cpu().numpy()
    for i in range(B):
        zref = mgp(x[i])
        assert np.linalg.norm(z[i] - zref) / np.linalg.norm(zref) < 2e-4
    b = np.zeros((B, ny, nx), dtype=np.complex128)
    for i, (jy, jx) in enumerate([(ny // 2, nx // 2), (40, 100), (120, 200)]):
        b[i, jy, jx] = 1.0
    xs, st = helm.fgmres_solve(P, _c64(b), restart=10, rtol=1e-6, maxit=2000)
    xs = xs.cpu().numpy()
    for i in range(B):
        rel = np.linalg.norm(b[i] - op.A(xs[i])) / np.linalg.norm(b[i])
        assert st["status"][i] == 1 and rel <= 1e-6, (i, rel)
