"""GPU parity of the tcgen05 implicit-GEMM convolution against the oracle's
convolution ops, for every layer shape of the network and every mode.

Inputs and weights are rounded to BF16 on the host, so the oracle sees exactly the
GPU's operands.  Remaining error: FP32 accumulation (<= K u32 sum|w||x|, K <= 576)
plus the final BF16 rounding of y (half an ulp, 2^-8 relative); the raw FP32
accumulator is compared with the first term only.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cnn as ocnn

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_17486_gb300 as h
    return h


def _bf(a):
    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).float().numpy().astype(np.float64)


def _oracle(x_nchw, w, mode, taps):
    tp = ocnn.Tape({"w": w}, record=False)
    v = ocnn.Var(x_nchw)
    if taps == 1:
        return ocnn.conv1x1(tp, v, "w").a
    if mode in ("s1", "s2"):
        return ocnn.conv3x3(tp, v, "w", 1 if mode == "s1" else 2).a
    return ocnn.conv3x3_transposed(tp, v, "w", 2 if mode == "t2" else 1).a


CASES = [  # (cin, cout, taps, mode, H, W)
    (2, 16, 9, "s1", 20, 30), (2, 16, 9, "s2", 24, 36), (16, 16, 9, "s1", 17, 23), (16, 32, 9, "s2", 32, 26),
    (32, 32, 9, "s1", 9, 40), (32, 64, 9, "s2", 18, 18), (64, 64, 9, "s1", 12, 12), (64, 64, 9, "s2", 16, 10),
    (64, 64, 9, "t2", 6, 9), (64, 32, 9, "t2", 8, 8), (32, 16, 9, "t2", 10, 7), (64, 64, 9, "t1", 9, 9),
    (16, 96, 1, "s1", 15, 21), (96, 16, 1, "s1", 15, 21), (32, 192, 1, "s1", 9, 13), (192, 32, 1, "s1", 9, 13),
    (64, 384, 1, "s1", 7, 11), (384, 64, 1, "s1", 7, 11), (16, 16, 9, "s1", 144, 144),
    (16, 16, 9, "t2", 5, 11), (32, 32, 9, "t2", 9, 4), (32, 16, 9, "t2", 72, 72), (64, 32, 9, "t2", 36, 36),
    # rows too wide for one row's window: segments of MMA steps within a row (the first
    # encoder convolution and the last solver downsampling of the 2176^2 grid)
    (2, 16, 9, "s2", 6, 2176), (64, 64, 9, "s2", 8, 272),
]


@pytest.mark.parametrize("cin,cout,taps,mode,H,W", CASES)
def test_conv_matches_oracle(helm, cin, cout, taps, mode, H, W):
    rng = np.random.default_rng(cin * 1000 + cout + H)
    B = 2
    x = _bf(rng.standard_normal((B, cin, H, W)))
    if taps == 1:
        w = _bf(rng.standard_normal((cout, cin)) / np.sqrt(cin))
    elif mode in ("s1", "s2"):
        w = _bf(rng.standard_normal((cout, cin, 3, 3)) / np.sqrt(9 * cin))
    else:
        w = _bf(rng.standard_normal((cin, cout, 3, 3)) / np.sqrt(9 * cin))
    ref = _oracle(x, w, mode, taps)
    refabs = _oracle(np.abs(x), np.abs(w), mode, taps)
    Ho, Wo = ref.shape[2:]
    scale = rng.uniform(0.5, 1.5, cout)
    shift = rng.uniform(-0.5, 0.5, cout)
    add1 = _bf(rng.standard_normal((B, cout, Ho, Wo)))
    add2 = _bf(rng.standard_normal((1, cout, Ho, Wo)))
    dev = "cuda"
    xg = torch.tensor(x.transpose(0, 2, 3, 1).copy(), dtype=torch.bfloat16, device=dev)
    wg = torch.tensor(w, dtype=torch.float32, device=dev)
    sc = torch.tensor(scale, dtype=torch.float32, device=dev)
    sh = torch.tensor(shift, dtype=torch.float32, device=dev)
    a1 = torch.tensor(add1.transpose(0, 2, 3, 1).copy(), dtype=torch.bfloat16, device=dev)
    a2 = torch.tensor(add2.transpose(0, 2, 3, 1).copy(), dtype=torch.bfloat16, device=dev)
    y, yr = helm.conv_bf16(xg, wg, mode, sc, sh, act=True, add1=a1, add2=a2, raw=True)
    torch.cuda.synchronize()
    yr = yr.cpu().numpy().transpose(0, 3, 1, 2)
    y = y.float().cpu().numpy().transpose(0, 3, 1, 2)
    acc_bound = 600 * U32 * refabs + 1e-30
    assert np.all(np.abs(yr - ref) <= acc_bound), np.max(np.abs(yr - ref) / acc_bound)
    pre = scale[None, :, None, None] * ref + shift[None, :, None, None]
    full = np.logaddexp(0.0, pre) + add1 + add2
    bound = 2.0 ** -8 * np.abs(full) + scale[None, :, None, None] * acc_bound + 1e-6 * (1 + np.abs(full))
    assert np.all(np.abs(y - full) <= bound), np.max(np.abs(y - full) / bound)
