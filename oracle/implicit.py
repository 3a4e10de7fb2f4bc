"""Oracle: the implicit layer (Section 4.2, Eq. 14) and the Green's function of a
learned 3x3 kernel (Eq. 15), with their adjoints for back-propagation.

Test infrastructure only (see the package docstring).

Readings of Section 4.2 (the paper's maps are square; an m_y x m_x map, with m_y
rows and m_x columns, takes every size below per axis: 6m_y x 6m_x, 2m_y x 2m_x):
  * A channel's kernel K is a complex 3x3 array; its operator is the circular
    convolution (K_pad * x)[p] = sum_a K_pad[a] x[p - a] with K_pad holding
    K[a+1] at offset a in {-1,0,1}^2, wrapped into the corners of the grid.
  * Eq. (15) is evaluated on a periodic grid three times the expanded size
    (n6 = 6m for an m x m feature map, expanded size 2m), with the point source
    delta at the centre index 3m.  The quotient F(K)/(F(K)^2 + eps) is read as the
    least-squares (Tikhonov) form conj(F(K)) / (|F(K)|^2 + eps); the literal form
    is available with literal=True.  eps = 1e-5.
  * crop(G_K) keeps the 2m x 2m window of offsets -m..m-1 around the source and
    stores offset 0 at index 0 (ifftshift); G_hat = F(crop(G_K)).
  * Eq. (14) on an m x m channel: zero-pad to 2m x 2m (data at the top-left),
    multiply by G_hat in Fourier space, invert, and keep the top-left m x m block.
    This is the linear (non-periodic) convolution of x with the cropped G.
"""
from __future__ import annotations

import numpy as np

EPS = 1e-5  # Eq. (15)


def dims(m) -> tuple[int, int]:
    """(m_y, m_x) of a coarsest map given as a side m (square) or a pair."""
    if np.ndim(m) == 0:
        return int(m), int(m)
    my, mx = m
    return int(my), int(mx)


def kernel_pad(K: np.ndarray, n, nx: int | None = None) -> np.ndarray:
    """Place a 3x3 kernel at the corners of an n x n (or n x nx) periodic grid
    (offset 0 at [0,0]); K[a+1, b+1] is the tap at row offset a, column offset b."""
    ny, nx = (n, n) if nx is None else (n, nx)
    Kp = np.zeros((ny, nx), dtype=np.complex128)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            Kp[a % ny, b % nx] += K[a + 1, b + 1]
    return Kp


def greens_raw(K: np.ndarray, m, eps: float = EPS, literal: bool = False):
    """G_K of Eq. (15) on the 6m_y x 6m_x periodic grid (source at the centre),
    plus the intermediates needed by the backward pass."""
    my, mx = dims(m)
    Khat = np.fft.fft2(kernel_pad(K, 6 * my, 6 * mx))
    if literal:
        Hq = Khat / (Khat ** 2 + eps)
    else:
        Hq = np.conj(Khat) / (np.abs(Khat) ** 2 + eps)
    delta = np.zeros((6 * my, 6 * mx), dtype=np.complex128)
    delta[3 * my, 3 * mx] = 1.0
    Fdelta = np.fft.fft2(delta)
    G = np.fft.ifft2(Hq * Fdelta)
    return G, Khat, Hq, Fdelta


def crop_centre(G: np.ndarray, m) -> np.ndarray:
    """crop(G_K): offsets -m..m-1 around the centre 3m (per axis), offset 0 moved to
    index 0."""
    my, mx = dims(m)
    win = G[2 * my:4 * my, 2 * mx:4 * mx]
    return np.fft.ifftshift(win)


def uncrop_centre(Gc: np.ndarray, m) -> np.ndarray:
    """Adjoint of crop_centre (embed the window back into a zero 6m_y x 6m_x grid)."""
    my, mx = dims(m)
    G = np.zeros((6 * my, 6 * mx), dtype=np.complex128)
    G[2 * my:4 * my, 2 * mx:4 * mx] = np.fft.fftshift(Gc)
    return G


def greens_hat(K: np.ndarray, m, eps: float = EPS, literal: bool = False) -> np.ndarray:
    """G_hat_K = F(crop(G_K)) on the 2m_y x 2m_x expanded grid (Section 4.2)."""
    G = greens_raw(K, m, eps, literal)[0]
    return np.fft.fft2(crop_centre(G, m))


def implicit_apply(x: np.ndarray, Ghat: np.ndarray) -> np.ndarray:
    """Eq. (14) for one complex channel x [..., m_y, m_x]: F^{-1}(G_hat (.) F(pad(x))),
    cropped; G_hat is [2m_y, 2m_x]."""
    my, mx = x.shape[-2:]
    xp = np.zeros(x.shape[:-2] + (2 * my, 2 * mx), dtype=np.complex128)
    xp[..., :my, :mx] = x
    y = np.fft.ifft2(Ghat * np.fft.fft2(xp))
    return y[..., :my, :mx]


def implicit_adjoint(gy: np.ndarray, Ghat: np.ndarray) -> np.ndarray:
    """Adjoint of Eq. (14) in x: the same map with conj(G_hat)."""
    return implicit_apply(gy, np.conj(Ghat))


def implicit_grad_ghat(x: np.ndarray, gy: np.ndarray) -> np.ndarray:
    """Gradient of a real loss with respect to G_hat (complex-gradient convention
    g = dL/dRe + i dL/dIm), summed over the leading batch dimensions.

    y = crop(F^{-1}(G_hat . X_hat)); with W = G_hat . X_hat, grad_W = F^{-H} pad(gy)
    = F(pad(gy)) / n^2, and grad_G_hat = conj(X_hat) . grad_W.
    """
    my, mx = x.shape[-2:]
    n2 = (2 * my) * (2 * mx)
    xp = np.zeros(x.shape[:-2] + (2 * my, 2 * mx), dtype=np.complex128)
    xp[..., :my, :mx] = x
    gp = np.zeros_like(xp)
    gp[..., :my, :mx] = gy
    Xh = np.fft.fft2(xp)
    gW = np.fft.fft2(gp) / n2
    g = np.conj(Xh) * gW
    return g.reshape((-1, 2 * my, 2 * mx)).sum(axis=0)


def greens_backward(K: np.ndarray, m, g_ghat: np.ndarray, eps: float = EPS,
                    literal: bool = False) -> np.ndarray:
    """Chain rule from grad(G_hat) back to the complex 3x3 kernel K (returns the
    complex gradient dL/dRe K + i dL/dIm K).

    Steps, each the adjoint of a forward step of `greens_hat`:
      G_hat = F(Gc)                  -> g_Gc = F^H g_ghat
      Gc = crop(G)                   -> g_G  = uncrop(g_Gc)
      G = F^{-1}(Hq . Fdelta)        -> g_T  = F^{-H} g_G = F(g_G)/n6^2,  g_Hq = conj(Fdelta) . g_T
      Hq = conj(Kh)/(|Kh|^2 + eps)   -> Wirtinger: a = dHq/dKh = -conj(Kh)^2/(|Kh|^2+eps)^2,
                                        b = dHq/dconj(Kh) = eps/(|Kh|^2+eps)^2,
                                        g_Kh = g_Hq conj(a) + conj(g_Hq) b
      (literal form Hq = Kh/(Kh^2+eps): holomorphic, a = (eps - Kh^2)/(Kh^2+eps)^2, b = 0)
      Kh = F(K_pad)                  -> g_Kpad = F^H g_Kh
      K_pad = kernel_pad(K)          -> g_K[a+1,b+1] = g_Kpad[a mod n6, b mod n6]
    """
    my, mx = dims(m)
    n6y, n6x = 6 * my, 6 * mx
    _, Kh, Hq, Fdelta = greens_raw(K, m, eps, literal)
    n2 = (2 * my) * (2 * mx)
    g_Gc = np.fft.ifft2(g_ghat) * n2            # F^H = n^2 F^{-1}
    g_G = uncrop_centre(g_Gc, m)
    g_T = np.fft.fft2(g_G) / (n6y * n6x)        # F^{-H} = F / n^2
    g_Hq = np.conj(Fdelta) * g_T
    if literal:
        a = (eps - Kh ** 2) / (Kh ** 2 + eps) ** 2
        g_Kh = g_Hq * np.conj(a)
    else:
        den = (np.abs(Kh) ** 2 + eps) ** 2
        a = -np.conj(Kh) ** 2 / den
        b = eps / den
        g_Kh = g_Hq * np.conj(a) + np.conj(g_Hq) * b
    g_Kpad = np.fft.ifft2(g_Kh) * (n6y * n6x)   # F^H
    gK = np.zeros((3, 3), dtype=np.complex128)
    for a_ in (-1, 0, 1):
        for b_ in (-1, 0, 1):
            gK[a_ + 1, b_ + 1] = g_Kpad[a_ % n6y, b_ % n6x]
    return gK


def laplacian_plus_i() -> np.ndarray:
    """Initial implicit kernel L + iI (Section 5.3), L the 5-point Laplacian
    stencil [0 -1 0; -1 4 -1; 0 -1 0] (sign of -Delta_h, as in Eq. 3)."""
    L = np.array([[0, -1, 0], [-1, 4, -1], [0, -1, 0]], dtype=np.complex128)
    I = np.zeros((3, 3), dtype=np.complex128)
    I[1, 1] = 1.0
    return L + 1j * I
