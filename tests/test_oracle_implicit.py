"""Pins of the oracle's implicit layer and Green's function (Section 4.2, Eq. 14-15)
against re-convolution, closed forms, brute-force convolution and finite
differences (no GPU)."""
import numpy as np
import pytest

import synth
from oracle import implicit as imp


def _circconv(K, x):
    """Brute-force circular convolution (K_pad * x)[p] = sum_a K[a+1] x[p-a]."""
    n = x.shape[0]
    y = np.zeros_like(x, dtype=np.complex128)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            y += K[a + 1, b + 1] * np.roll(np.roll(x, a, axis=0), b, axis=1)
    return y


def test_kernel_hat_closed_form_for_laplacian_plus_shift():
    """K = L + c delta: F(K_pad) = 4 - 2cos(t1) - 2cos(t2) + c."""
    n = 12
    c = 0.3 + 1.0j
    K = imp.laplacian_plus_i().real.astype(complex)
    K[1, 1] += c
    Kh = np.fft.fft2(imp.kernel_pad(K, n))
    t = 2 * np.pi * np.arange(n) / n
    ref = 4 - 2 * np.cos(t)[:, None] - 2 * np.cos(t)[None, :] + c
    assert np.allclose(Kh, ref, atol=1e-13)


def test_green_reconvolution_identity_with_eps_zero():
    """With eps = 0 on the uncropped periodic 6m grid, K * (G * x) = x exactly."""
    m = 4
    n6 = 6 * m
    K = imp.laplacian_plus_i()
    K = K + 0.1 * synth.random_complex((3, 3), 1)
    G, *_ = imp.greens_raw(K, m, eps=0.0)
    # G is the response to a source at the centre 3m: shift it back to offset 0
    G0 = np.roll(np.roll(G, -3 * m, axis=0), -3 * m, axis=1)
    x = synth.random_complex((n6, n6), 2)
    Gx = np.fft.ifft2(np.fft.fft2(G0) * np.fft.fft2(x))
    assert np.allclose(_circconv(K, Gx), x, atol=1e-12)


def test_green_reconvolution_deviation_bounded_by_eps():
    """At eps = 1e-5 and the L + iI initialisation (|K_hat| >= 1), the periodic
    re-convolution deviates from the identity by at most eps / (|K_hat|^2 + eps)."""
    m = 4
    K = imp.laplacian_plus_i()
    G, Kh, *_ = imp.greens_raw(K, m, eps=imp.EPS)
    G0 = np.roll(np.roll(G, -3 * m, axis=0), -3 * m, axis=1)
    x = synth.random_complex((6 * m, 6 * m), 3)
    y = _circconv(K, np.fft.ifft2(np.fft.fft2(G0) * np.fft.fft2(x)))
    bound = (imp.EPS / (np.abs(Kh) ** 2 + imp.EPS)).max()
    assert np.abs(Kh).min() >= 1.0 - 1e-12
    assert np.linalg.norm(y - x) <= bound * np.linalg.norm(x) * (1 + 1e-9)


def test_implicit_apply_is_linear_convolution_with_cropped_green():
    """Eq. (14) with the 2m zero padding equals the direct (non-periodic) convolution
    of x with G restricted to offsets -m..m-1."""
    m = 5
    K = imp.laplacian_plus_i() + 0.2 * synth.random_complex((3, 3), 4)
    Ghat = imp.greens_hat(K, m)
    Gc = np.fft.ifft2(Ghat)                     # offset d stored at index d mod 2m
    x = synth.random_complex((m, m), 5)
    y = imp.implicit_apply(x, Ghat)
    ref = np.zeros((m, m), complex)
    for i in range(m):
        for j in range(m):
            for p in range(m):
                for q in range(m):
                    ref[i, j] += Gc[(i - p) % (2 * m), (j - q) % (2 * m)] * x[p, q]
    assert np.allclose(y, ref, atol=1e-13)
    # and G itself approximately inverts K near the source (discrete Green's function)
    G, *_ = imp.greens_raw(K, m)
    c = 3 * m
    KG = _circconv(K, G)
    delta = np.zeros_like(KG)
    delta[c, c] = 1
    assert np.abs(KG - delta).max() < 1e-4


def test_implicit_adjoint_identity():
    m = 6
    K = imp.laplacian_plus_i() + 0.3 * synth.random_complex((3, 3), 7)
    Ghat = imp.greens_hat(K, m)
    x = synth.random_complex((m, m), 8)
    y = synth.random_complex((m, m), 9)
    lhs = np.vdot(imp.implicit_apply(x, Ghat), y)
    rhs = np.vdot(x, imp.implicit_adjoint(y, Ghat))
    assert np.isclose(lhs, rhs, rtol=1e-12)


@pytest.mark.parametrize("literal", [False, True])
def test_kernel_gradient_matches_finite_differences(literal):
    m = 4
    K = imp.laplacian_plus_i() + 0.3 * synth.random_complex((3, 3), 10)
    x = synth.random_complex((2, m, m), 11)
    w = synth.random_complex((2, m, m), 12)

    def loss(Kc):
        y = imp.implicit_apply(x, imp.greens_hat(Kc, m, literal=literal))
        return float(np.real(np.vdot(w, y)))   # real, linear in y: dL/dy = w

    g_gh = imp.implicit_grad_ghat(x, w)
    gK = imp.greens_backward(K, m, g_gh, literal=literal)
    h = 1e-6
    for idx in [(0, 0), (1, 1), (2, 1)]:
        for part, unit in (("re", 1.0), ("im", 1j)):
            Kp = K.copy(); Kp[idx] += h * unit
            Km = K.copy(); Km[idx] -= h * unit
            fd = (loss(Kp) - loss(Km)) / (2 * h)
            an = gK[idx].real if part == "re" else gK[idx].imag
            assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-8), (idx, part, fd, an)
