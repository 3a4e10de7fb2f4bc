"""GPU tests of the captured solver plans used for mixed-size serving: a plan's graph-
replayed solve equals the eager helm_fgmres_solve bit for bit (V-cycle only and with the
network, whose captured cycles run it on the whole batch and zero the outputs of
right-hand sides that fell back), after an in-place problem update as well; a plan
refuses to run once the network's parameters or encodings no longer match it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_17486_gb300 as h
    return h


def _kappa(n, abl, seed):
    return synth.layered_grf_kappa(n, abl, seed=seed).astype(np.float32)


def _net(helm):
    import os
    from paper_2306_17486_gb300 import train as T
    net = helm.Cnn(skip_threshold=256)
    T.load_weights(net, os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                     "paper_2306_17486_gb300", "weights", "cnn_grf_multiscale.npz"))
    return net


@pytest.mark.parametrize("with_net", [False, True], ids=["mg", "cnn"])
def test_plan_solve_matches_eager_bitwise(helm, with_net):
    n, abl, B = 96, 16, 4
    N = n + 2 * abl
    k1, k2 = _kappa(n, abl, 3), _kappa(n, abl, 4)
    oh1, oh2 = 2 * np.pi / 10 / k1.max(), 2 * np.pi / 10 / k2.max()
    kt1 = torch.tensor(k1, device="cuda")
    kt2 = torch.tensor(k2, device="cuda")
    net = _net(helm) if with_net else None
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        p = helm.Problem(kt1, abl, oh1, levels=3)
        if net is not None:
            net.set_problem(p)
        plan = helm.SolverPlan(p, B, cnn=net, restart=10, rtol=1e-6, maxit=600, stream=st)
        for kt, oh, seed in ((kt1, oh1, 5), (kt2, oh2, 6)):
            if kt is kt2:
                helm.problem_update(p, kt, oh)
                if net is not None:
                    net.set_problem(p)
            b = torch.tensor(synth.random_point_sources(N, abl, B, seed=seed), dtype=torch.complex64, device="cuda")
            plan.b.copy_(b)
            st_plan = plan.solve()
            x_eager, st_eager = helm.fgmres_solve(p, b, cnn=net, restart=10, rtol=1e-6, maxit=600)
            torch.cuda.synchronize()
            assert (st_plan["status"] == 1).all(), st_plan
            assert np.array_equal(st_plan["iters"], st_eager["iters"]), (st_plan, st_eager)
            assert torch.equal(plan.x, x_eager)
            # a fresh problem built from the updated kappa gives the same solution
            if kt is kt2:
                p2 = helm.Problem(kt2, abl, oh2, levels=3)
                if net is not None:
                    net.set_problem(p2)
                x2, _ = helm.fgmres_solve(p2, b, cnn=net, restart=10, rtol=1e-6, maxit=600)
                torch.cuda.synchronize()
                assert torch.equal(x2, x_eager)
                if net is not None:
                    net.set_problem(p)
    assert helm.device_errors() == 0


def test_plan_refuses_stale_network(helm):
    n, abl, B = 96, 16, 2
    k = _kappa(n, abl, 7)
    kt = torch.tensor(k, device="cuda")
    net = _net(helm)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        p = helm.Problem(kt, abl, 2 * np.pi / 10 / k.max(), levels=3)
        with pytest.raises(helm.HelmError, match="encodings"):
            helm.SolverPlan(p, B, cnn=net, stream=st)      # no set_problem yet
        net.set_problem(p)
        plan = helm.SolverPlan(p, B, cnn=net, stream=st)
        helm.problem_update(p, kt, 2 * np.pi / 10 / k.max())
        with pytest.raises(helm.HelmError, match="encodings"):
            plan.solve()                                   # problem updated, encodings stale
        net.set_problem(p)
        plan.solve()
        net.set_params(net.params.clone())
        with pytest.raises(helm.HelmError, match="parameters changed"):
            plan.solve()
