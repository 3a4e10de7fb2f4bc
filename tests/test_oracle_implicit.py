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


# ---- rectangular coarsest maps (m_y x m_x): every size of Eq. (14)-(15) per axis -----

def _greens_hat_brute(K, my, mx, eps=imp.EPS):
    """G_hat of an m_y x m_x map with explicit DFT sums and no FFT: K_hat on the
    6m_y x 6m_x periodic grid from the nine taps, the Tikhonov quotient, G at the
    2m_y x 2m_x offsets around the source, then the 2D DFT of the cropped window."""
    ny, nx = 6 * my, 6 * mx
    u = np.arange(ny)[:, None]
    v = np.arange(nx)[None, :]
    Kh = np.zeros((ny, nx), complex)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            Kh += K[a + 1, b + 1] * np.exp(-2j * np.pi * (a * u / ny + b * v / nx))
    H = np.conj(Kh) / (np.abs(Kh) ** 2 + eps)
    dy = [i if i < my else i - 2 * my for i in range(2 * my)]
    dx = [j if j < mx else j - 2 * mx for j in range(2 * mx)]
    Gc = np.zeros((2 * my, 2 * mx), complex)
    for i, di in enumerate(dy):
        for j, dj in enumerate(dx):
            # the source sits at (3m_y, 3m_x): G there + offset d is the inverse DFT at d
            Gc[i, j] = (H * np.exp(2j * np.pi * (u * di / ny + v * dj / nx))).sum() / (ny * nx)
    p = np.arange(2 * my)[:, None]
    q = np.arange(2 * mx)[None, :]
    Gh = np.zeros_like(Gc)
    for i in range(2 * my):
        for j in range(2 * mx):
            Gh += Gc[i, j] * np.exp(-2j * np.pi * (p * i / (2 * my) + q * j / (2 * mx)))
    return Gh


def test_rectangular_green_hat_matches_brute_force_sums():
    K = imp.laplacian_plus_i() + 0.25 * synth.random_complex((3, 3), 20)
    for my, mx in ((2, 3), (3, 2)):
        assert np.allclose(imp.greens_hat(K, (my, mx)), _greens_hat_brute(K, my, mx), atol=1e-12)


def test_rectangular_green_and_layer_transpose_with_the_kernel():
    """Transposing the kernel transposes G_hat of the transposed map, and Eq. (14) on
    the transposed input gives the transposed output: an exchanged axis fails here."""
    K = imp.laplacian_plus_i() + 0.3 * synth.random_complex((3, 3), 21)
    K[0, 1] += 0.4    # an asymmetric kernel: K != K^T
    my, mx = 3, 5
    Gh = imp.greens_hat(K, (my, mx))
    assert Gh.shape == (2 * my, 2 * mx)
    GhT = imp.greens_hat(K.T, (mx, my))
    assert np.allclose(GhT, Gh.T, atol=1e-13)
    assert not np.allclose(imp.greens_hat(K, (mx, my)), GhT, atol=1e-6)
    x = synth.random_complex((2, my, mx), 22)
    y = imp.implicit_apply(x, Gh)
    yT = imp.implicit_apply(np.swapaxes(x, -1, -2), GhT)
    assert np.allclose(yT, np.swapaxes(y, -1, -2), atol=1e-13)


def test_rectangular_implicit_apply_is_linear_convolution_with_cropped_green():
    my, mx = 3, 5
    K = imp.laplacian_plus_i() + 0.2 * synth.random_complex((3, 3), 23)
    Ghat = imp.greens_hat(K, (my, mx))
    Gc = np.fft.ifft2(Ghat)
    x = synth.random_complex((my, mx), 24)
    y = imp.implicit_apply(x, Ghat)
    ref = np.zeros((my, mx), complex)
    for i in range(my):
        for j in range(mx):
            for p in range(my):
                for q in range(mx):
                    ref[i, j] += Gc[(i - p) % (2 * my), (j - q) % (2 * mx)] * x[p, q]
    assert np.allclose(y, ref, atol=1e-13)
    # the uncropped G inverts K on the periodic grid up to the eps regularisation
    G, *_ = imp.greens_raw(K, (my, mx))
    KG = np.zeros_like(G)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            KG += K[a + 1, b + 1] * np.roll(np.roll(G, a, axis=0), b, axis=1)
    delta = np.zeros_like(KG)
    delta[3 * my, 3 * mx] = 1
    assert np.abs(KG - delta).max() < 1e-4


def test_rectangular_adjoint_and_kernel_gradient():
    my, mx = 3, 4
    K = imp.laplacian_plus_i() + 0.3 * synth.random_complex((3, 3), 25)
    Ghat = imp.greens_hat(K, (my, mx))
    x = synth.random_complex((2, my, mx), 26)
    w = synth.random_complex((2, my, mx), 27)
    assert np.isclose(np.vdot(imp.implicit_apply(x, Ghat), w), np.vdot(x, imp.implicit_adjoint(w, Ghat)),
                      rtol=1e-12)

    def loss(Kc):
        return float(np.real(np.vdot(w, imp.implicit_apply(x, imp.greens_hat(Kc, (my, mx))))))

    gK = imp.greens_backward(K, (my, mx), imp.implicit_grad_ghat(x, w))
    h = 1e-6
    for idx in [(0, 1), (1, 1), (2, 0)]:
        for unit in (1.0, 1j):
            Kp = K.copy(); Kp[idx] += h * unit
            Km = K.copy(); Km[idx] -= h * unit
            fd = (loss(Kp) - loss(Km)) / (2 * h)
            an = gK[idx].real if unit == 1.0 else gK[idx].imag
            assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-8), (idx, unit, fd, an)
