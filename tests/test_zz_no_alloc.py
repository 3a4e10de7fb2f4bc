"""GPU test of the allocation-free V-cycle entry point (helm_slmg_vcycle_static): its
output equals the workspace V-cycle's on the same input, on two calls in a row (the
static scratch is reused with whatever the previous call left in it), and a batch
whose scratch exceeds the fixed array is rejected before anything is launched.

Tolerance: both calls run the same kernels on the same data, so they agree to
rounding-order effects at most; bound 1e-6 of the output's largest entry."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_17486_gb300 as h
    return h


def _problem(helm, n, abl, levels, seed):
    kap = synth.layered_kappa(n, abl, seed=seed)
    kt = torch.tensor(kap, dtype=torch.float32, device=DEV)
    return helm.Problem(kt, abl, 2 * np.pi / 10 / float(kap.max()), levels=levels)


@pytest.mark.parametrize("n,abl,levels,batch", [(256, 16, 4, 3), (512, 32, 4, 2), (96, 16, 3, 5)])
def test_static_vcycle_matches_workspace_vcycle(helm, n, abl, levels, batch):
    P = _problem(helm, n, abl, levels, seed=1)
    N = n + 2 * abl
    r1 = torch.tensor(synth.random_complex((batch, N, N), seed=7), dtype=torch.complex64, device=DEV)
    r2 = torch.tensor(synth.random_complex((batch, N, N), seed=8), dtype=torch.complex64, device=DEV)
    for r in (r1, r2):   # two different inputs back to back through the same scratch
        z_ref = helm.slmg_vcycle(P, r)
        z_a = helm.slmg_vcycle_static(P, r)
        z_b = helm.slmg_vcycle_static(P, r)
        torch.cuda.synchronize()
        scale = z_ref.abs().max().item()
        assert scale > 0
        for z in (z_a, z_b):
            err = (z - z_ref).abs().max().item()
            assert err <= 1e-6 * scale, (n, batch, err, scale)
    assert helm.device_errors() == 0


def test_static_vcycle_rejects_oversized_batch(helm):
    P = _problem(helm, 512, 32, 4, seed=2)
    r = torch.zeros((64, 576, 576), dtype=torch.complex64, device=DEV)
    z = torch.full_like(r, complex(3.0, 3.0))
    with pytest.raises(helm.HelmError, match="static scratch holds"):
        helm.slmg_vcycle_static(P, r, z)
    torch.cuda.synchronize()
    assert bool((z == complex(3.0, 3.0)).all())   # nothing was launched
