"""GPU tests of the launch-shape tuning table: every tuned work-unit shape of the
convolution and inverted-bottleneck kernels gives the network output of the heuristic
shapes bit for bit (each output pixel is reduced in the same order whatever the unit
it falls in), and the autotuner's entries round-trip through its JSON file."""
import os

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


def _setup(helm, n, abl, B, seed=11):
    from paper_2306_17486_gb300 import train as T
    N = n + 2 * abl
    k = torch.tensor(synth.layered_grf_kappa(n, abl, seed=seed), dtype=torch.float32, device="cuda")
    p = helm.Problem(k, abl, 2 * np.pi / 10 / float(k.max()), levels=2)
    net = helm.Cnn(skip_threshold=256)
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    T.load_weights(net, os.path.join(here, "paper_2306_17486_gb300", "weights", "cnn_grf_multiscale.npz"))
    net.set_problem(p)
    g = torch.Generator().manual_seed(seed)
    r = torch.complex(torch.randn(B, N, N, generator=g), torch.randn(B, N, N, generator=g)).to(torch.complex64).cuda()
    return N, p, net, r


@pytest.mark.parametrize("n,abl,B", [(256, 16, 3), (160, 16, 2)])
def test_tuned_shapes_bitwise(helm, n, abl, B):
    from paper_2306_17486_gb300.autotune import level_heights
    N, p, net, r = _setup(helm, n, abl, B)
    helm.tune_clear()
    ref = net.apply(p, r)
    torch.cuda.synchronize()
    for knob, values in (("conv_rows", (1, 2, 3, 8, 32)), ("ib_sh", (4, 8, 12, 40, 1000))):
        for v in values:
            for h in level_heights(N):
                helm.tune_set(knob, h, B, v)
            out = net.apply(p, r)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), (knob, v)
        helm.tune_clear()
    assert helm.device_errors() == 0


def test_autotune_roundtrip(helm, tmp_path):
    from paper_2306_17486_gb300 import autotune
    helm.tune_clear()
    res = autotune.tune_grid(288, 16, 2, reps=3)
    assert res["ms_tuned"] > 0 and res["ms_heuristic"] > 0
    for knob, h, v in res["entries"]:
        assert helm.tune_get(knob, h, 2) == v
    path = str(tmp_path / "shapes.json")
    autotune.save([res], path)
    helm.tune_clear()
    assert autotune.apply(path, grids={(288, 2)}) == len(res["entries"])
    for knob, h, v in res["entries"]:
        assert helm.tune_get(knob, h, 2) == v
    assert autotune.apply(path, grids={(576, 2)}) == 0
    helm.tune_clear()
