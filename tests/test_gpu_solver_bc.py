"""GPU parity of the Neumann and Sommerfeld boundary conditions (ghost values c u_b
folded into the mass term of every level; Section 3.4 remark, Section 3.1) against the
FP64 oracle, through the C ABI.  Tolerances as for the Dirichlet problems: the setup
fields are computed in FP64 and rounded once, the stencil within 8u of its operand
scale, the V-cycle within 2e-4, FGMRES judged by the oracle's true FP64 residual."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import fgmres as ofg
from oracle import helmholtz as ohz
from oracle import multigrid as omg

pytestmark = pytest.mark.gpu
U = 2.0 ** -24
DEV = "cuda:0"


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_17486_gb300 as h
    return h


def _mk(helm, ny, nx, abl, levels, bc, seed=0, gamma0=0.0):
    if ny == nx:
        kappa = synth.grf_kappa(ny - 2 * abl, abl, 6.0, seed)
    else:
        rng = np.random.default_rng(seed)
        kappa = 0.25 + 0.75 * rng.random((ny, nx))
    kappa32 = kappa.astype(np.float32).astype(np.float64)
    oh = ohz.omega_h_for_ppw(kappa32.max())
    P = helm.Problem(torch.tensor(kappa32, dtype=torch.float32, device=DEV), abl, oh, gamma0=gamma0,
                     levels=levels, bc=bc)
    op = ohz.Problem(kappa32, abl, omega_h=oh, gamma0=gamma0, bc=bc)
    return P, op


def _c64(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.complex64, device=DEV)


def _q(a):
    return a.astype(np.complex64).astype(np.complex128)


CASES = [(48, 48, 8, 3, "neumann"), (48, 48, 8, 3, "sommerfeld"), (64, 96, 0, 3, "sommerfeld"),
         (64, 64, 0, 3, "neumann")]


@pytest.mark.parametrize("ny,nx,abl,levels,bc", CASES)
def test_bc_setup_fields_match_oracle(helm, ny, nx, abl, levels, bc):
    P, op = _mk(helm, ny, nx, abl, levels, bc, seed=1, gamma0=0.01)
    mg = omg.SLMultigrid(op, levels)
    mA = P.field("mass_A").cpu().numpy()
    assert np.all(np.abs(mA - op.mass_A) <= 2 * U * np.abs(op.mass_A) + 1e-30)
    # the boundary ring carries the condition's term (corners twice)
    assert abs(mA[0, 0].real - op.mass_A[0, 0].real) <= 4 * U * abs(op.mass_A[0, 0])
    for l in range(levels):
        m = P.field("mass_SL", l).cpu().numpy()
        assert np.all(np.abs(m - mg.mass[l]) <= 4 * U * np.abs(mg.mass[l]) + 1e-7), l
        d = P.field("dinv_SL", l).cpu().numpy()
        dref = 0.8 / (4.0 - mg.mass[l])
        assert np.all(np.abs(d - dref) <= 4 * U * np.abs(dref)), l


@pytest.mark.parametrize("ny,nx,abl,levels,bc", CASES)
def test_bc_apply_and_residual_match_oracle(helm, ny, nx, abl, levels, bc):
    P, op = _mk(helm, ny, nx, abl, levels, bc, seed=2)
    x = _q(synth.random_complex((2, ny, nx), 3))
    y = helm.helmholtz_apply(P, _c64(x)).cpu().numpy()
    ref = op.A(x)
    xp = np.pad(np.abs(x), ((0, 0), (1, 1), (1, 1)))
    scale = np.abs(4 - op.mass_A) * np.abs(x) + xp[:, :-2, 1:-1] + xp[:, 2:, 1:-1] + xp[:, 1:-1, :-2] + xp[:, 1:-1, 2:]
    assert np.all(np.abs(y - ref) <= 8 * U * scale)
    # the FP64 residual uses the FP64 copy of the same mass term
    b = _q(synth.random_complex((2, ny, nx), 5))
    xd = synth.random_complex((2, ny, nx), 6)
    r, _ = helm.helmholtz_residual_fp64(P, _c64(b), torch.tensor(xd, dtype=torch.complex128, device=DEV))
    rref = b - op.A(xd)
    assert np.all(np.abs(r.cpu().numpy() - rref) <= 2 * U * np.abs(rref) + 1e-13 * (np.abs(b) + 10 * np.abs(xd)))


@pytest.mark.parametrize("ny,nx,abl,levels,bc", CASES)
def test_bc_vcycle_matches_oracle(helm, ny, nx, abl, levels, bc):
    P, op = _mk(helm, ny, nx, abl, levels, bc, seed=7)
    mg = omg.SLMultigrid(op, levels, coarse="gmres", coarse_iters=10)
    r = _q(synth.random_complex((2, ny, nx), 8))
    z = helm.slmg_vcycle(P, _c64(r)).cpu().numpy()
    for i in range(2):
        zref = mg(r[i])
        err = np.linalg.norm(z[i] - zref) / np.linalg.norm(zref)
        assert err < 2e-4, err


@pytest.mark.parametrize("n,abl,bc", [(96, 16, "neumann"), (96, 0, "sommerfeld"), (96, 16, "sommerfeld")])
def test_bc_fgmres_converges_like_the_oracle(helm, n, abl, bc):
    """FGMRES(10) with the SL V-cycle to 1e-6: every RHS converges with a true FP64
    residual <= 1e-6 of the oracle's operator, in about the oracle's iteration count.
    (A closed Neumann box without a layer and without attenuation is a lossless cavity,
    near resonance at these frequencies; it is not a test case.)"""
    P, op = _mk(helm, n, n, abl, 3, bc, seed=3)
    b = synth.random_point_sources(n, abl, 2, seed=5)
    x, st = helm.fgmres_solve(P, _c64(b), restart=10, rtol=1e-6, maxit=2000)
    xs = x.cpu().numpy()
    mg = omg.SLMultigrid(op, 3)
    for i in range(2):
        assert st["status"][i] == 1, st
        true = np.linalg.norm(b[i] - op.A(xs[i])) / np.linalg.norm(b[i])
        assert true <= 1e-6 and abs(true - st["rel_res_true"][i]) <= 1e-9
        _, res = ofg.fgmres(op.A, b[i], np.zeros_like(b[i]), mg, 10, 1e-6, 2000)
        assert res.converged and st["iters"][i] <= 1.25 * res.iters + 5, (st["iters"][i], res.iters)
