"""GPU test of the allocation-free V-cycle entry point (helm_slmg_vcycle_static).

Some callers cannot allocate device memory or hand the library a workspace: a
preconditioner callback of an external Krylov package receives only its input and
output vectors, and a cudaMalloc inside such a callback would synchronise the whole
device on every iteration.  The static entry point serves them; this file checks
that it computes exactly what the workspace V-cycle computes:

* its output equals the workspace V-cycle's on the same input, bit for bit (both run
  the same kernels in the same order on the same data), on two calls in a row, so
  the second call starts from whatever the first left in the shared scratch;
* on the coarsest-solve path that keeps its Krylov basis in the scratch (GMRES with a
  step count other than the cluster kernel's 10) as well as on the cluster path;
* a call allocates nothing: neither PyTorch's allocator nor the device's free memory
  changes across it;
* a batch whose scratch exceeds the fixed array is rejected before anything runs.

The file is named so that pytest collects it last."""
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


def _problem(helm, n, abl, levels, seed, **mg):
    kap = synth.layered_kappa(n, abl, seed=seed)
    kt = torch.tensor(kap, dtype=torch.float32, device=DEV)
    return helm.Problem(kt, abl, 2 * np.pi / 10 / float(kap.max()), levels=levels, **mg)


@pytest.mark.parametrize("n,abl,levels,batch,coarse_iters", [
    (256, 16, 4, 3, 10), (512, 32, 4, 2, 10), (96, 16, 3, 5, 10),
    (256, 16, 4, 3, 6), (96, 16, 3, 2, 12)])
def test_static_vcycle_matches_workspace_vcycle(helm, n, abl, levels, batch, coarse_iters):
    P = _problem(helm, n, abl, levels, seed=1, coarse_iters=coarse_iters)
    N = n + 2 * abl
    r1 = torch.tensor(synth.random_complex((batch, N, N), seed=7), dtype=torch.complex64, device=DEV)
    r2 = torch.tensor(synth.random_complex((batch, N, N), seed=8), dtype=torch.complex64, device=DEV)
    for r in (r1, r2):   # two different inputs back to back through the same scratch
        z_ref = helm.slmg_vcycle(P, r)
        z_a = helm.slmg_vcycle_static(P, r)
        z_b = helm.slmg_vcycle_static(P, r)
        torch.cuda.synchronize()
        assert z_ref.abs().max().item() > 0
        assert torch.equal(z_a, z_ref), (n, batch, coarse_iters, (z_a - z_ref).abs().max().item())
        assert torch.equal(z_b, z_ref)
    assert helm.device_errors() == 0


def test_static_vcycle_allocates_nothing(helm):
    P = _problem(helm, 256, 16, 4, seed=3)
    r = torch.tensor(synth.random_complex((2, 288, 288), seed=9), dtype=torch.complex64, device=DEV)
    z = torch.empty_like(r)
    helm.slmg_vcycle_static(P, r, z)       # first call on the device: address set-up
    torch.cuda.synchronize()
    alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    helm.slmg_vcycle_static(P, r, z)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_vcycle_rejects_oversized_batch(helm):
    P = _problem(helm, 512, 32, 4, seed=2)
    r = torch.zeros((64, 576, 576), dtype=torch.complex64, device=DEV)
    z = torch.full_like(r, complex(3.0, 3.0))
    with pytest.raises(helm.HelmError, match="static scratch holds"):
        helm.slmg_vcycle_static(P, r, z)
    torch.cuda.synchronize()
    assert bool((z == complex(3.0, 3.0)).all())   # nothing was launched
