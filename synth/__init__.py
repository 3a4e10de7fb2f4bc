"""Seeded synthetic inputs shared by the FP64 oracle tests and the CUDA path.

This module draws random numbers and shapes them into inputs; it contains none of
the method's arithmetic (no operator, no multigrid, no Krylov step, no network).
Both sides receive exactly the arrays produced here.

The paper trains and tests on slowness models derived from image datasets
(Section 4.3, "Slowness Model Datasets"): images resized, smoothed slightly by a
Gaussian kernel and normalised to [0.25, 1].  Those datasets are not available,
so seeded Gaussian random fields and layered models with the same value range
and smoothing stand in for them.
"""
from __future__ import annotations

import numpy as np
from scipy.ndimage import gaussian_filter

KAPPA_MIN = 0.25   # Section 4.3: slowness normalised to [0.25, 1]
KAPPA_MAX = 1.0


def _to_range(f: np.ndarray, lo: float = KAPPA_MIN, hi: float = KAPPA_MAX) -> np.ndarray:
    f = f - f.min()
    span = f.max()
    if span <= 0:
        return np.full_like(f, 0.5 * (lo + hi))
    return lo + (hi - lo) * (f / span)


def _embed_abl(interior: np.ndarray, abl: int) -> np.ndarray:
    """Edge-replicate an n x n interior field into an (n+2L) x (n+2L) grid."""
    return np.pad(interior, abl, mode="edge")


def grf_kappa(n: int, abl: int, ell: float = 8.0, seed: int = 0) -> np.ndarray:
    """Gaussian random field slowness on the n x n interior, values in [0.25, 1].

    White N(0,1) noise filtered by a Gaussian of standard deviation ell/sqrt(2)
    cells (covariance exp(-d^2 / (2 ell^2))), min-max mapped to [0.25, 1] and
    edge-replicated into the absorbing layer.  Returns float64 [N][N].
    """
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n, n))
    f = gaussian_filter(w, sigma=ell / np.sqrt(2.0), mode="wrap")
    return _embed_abl(_to_range(f), abl)


def layered_kappa(n: int, abl: int, interfaces: int = 8, sigma: float = 2.0,
                  seed: int = 1) -> np.ndarray:
    """Piecewise-smooth layered slowness: `interfaces` random horizontal interfaces,
    layer values uniform in [0.25, 1], Gaussian-smoothed with sigma cells and
    renormalised to [0.25, 1].  Returns float64 [N][N] including the layer."""
    rng = np.random.default_rng(seed)
    depths = np.sort(rng.integers(1, n, size=interfaces))
    values = rng.uniform(KAPPA_MIN, KAPPA_MAX, size=interfaces + 1)
    col = np.empty(n)
    edges = np.concatenate([[0], depths, [n]])
    for k in range(interfaces + 1):
        col[edges[k]:edges[k + 1]] = values[k]
    f = np.repeat(col[:, None], n, axis=1)
    f = gaussian_filter(f, sigma=sigma, mode="nearest")
    return _embed_abl(_to_range(f), abl)


def layered_grf_kappa(n: int, abl: int, seed: int = 0) -> np.ndarray:
    """0.5 * layered + 0.5 * GRF, renormalised to [0.25, 1]."""
    a = layered_kappa(n, 0, seed=seed)
    b = grf_kappa(n, 0, seed=seed + 7919)
    return _embed_abl(_to_range(0.5 * a + 0.5 * b), abl)


def salt_kappa(n: int, abl: int, seed: int = 0) -> np.ndarray:
    """Out-of-distribution stand-in for a salt-dome model: a smooth layered background
    (slowness decreasing with depth, i.e. velocity increasing, with 6 random
    interfaces) holding a high-velocity body (slowness 0.25) bounded by a random smooth
    closed curve, Gaussian-smoothed with sigma 1 and renormalised to [0.25, 1].  Sharper
    contrast and larger features than the training fields.  Returns float64 [N][N]."""
    rng = np.random.default_rng(seed)
    y = np.linspace(0.0, 1.0, n)[:, None] * np.ones((1, n))
    depths = np.sort(rng.uniform(0.1, 0.9, size=6))
    values = np.sort(rng.uniform(0.45, 1.0, size=7))[::-1]
    f = np.full((n, n), values[0])
    for d, v in zip(depths, values[1:]):
        f = np.where(y >= d, v, f)
    yy, xx = np.mgrid[0:n, 0:n] / (n - 1.0)
    cy, cx = rng.uniform(0.35, 0.55), rng.uniform(0.35, 0.65)
    th = np.arctan2(yy - cy, xx - cx)
    rad = 0.18 + 0.04 * np.sin(3 * th + rng.uniform(0, 2 * np.pi)) + 0.03 * np.cos(5 * th + rng.uniform(0, 2 * np.pi))
    body = np.hypot(yy - cy, (xx - cx) * 0.7) < rad
    f = np.where(body, KAPPA_MIN, f)
    f = gaussian_filter(f, sigma=1.0, mode="nearest")
    return _embed_abl(_to_range(f), abl)


def rect_kappa(h: int, w: int, abl: int, seed: int = 0, kind: str = "grf") -> np.ndarray:
    """A rectangular model: an h x w interior (rows x columns) cut from the top-left of a
    square model of side max(h, w) ('grf', 'layered_grf' or 'salt' above), edge-replicated
    into the absorbing layer.  Returns float64 [h + 2 abl][w + 2 abl]."""
    n = max(h, w)
    make = {"grf": lambda: grf_kappa(n, 0, seed=seed), "layered_grf": lambda: layered_grf_kappa(n, 0, seed=seed),
            "salt": lambda: salt_kappa(n, 0, seed=seed)}[kind]
    return _embed_abl(make()[:h, :w], abl)


def rect_point_sources(h: int, w: int, abl: int, count: int, seed: int) -> np.ndarray:
    """`count` unit point sources at seeded positions inside the interior of an
    (h + 2 abl) x (w + 2 abl) grid, one per right-hand side: complex128 [count][H][W]."""
    rng = np.random.default_rng(seed)
    b = np.zeros((count, h + 2 * abl, w + 2 * abl), dtype=np.complex128)
    for i in range(count):
        b[i, abl + rng.integers(0, h), abl + rng.integers(0, w)] = 1.0
    return b


def centre_source(N: int) -> np.ndarray:
    """h^2-scaled right-hand side of a unit point source at the grid centre:
    h^2 g = 1 at node (N//2, N//2).  complex128 [N][N]."""
    b = np.zeros((N, N), dtype=np.complex128)
    b[N // 2, N // 2] = 1.0
    return b


def random_point_sources(N: int, abl: int, count: int, seed: int) -> np.ndarray:
    """`count` unit point sources at seeded positions drawn uniformly over the
    interior (non-absorbing) nodes.  complex128 [count][N][N]."""
    rng = np.random.default_rng(seed)
    n = N - 2 * abl
    b = np.zeros((count, N, N), dtype=np.complex128)
    iy = rng.integers(abl, abl + n, size=count)
    ix = rng.integers(abl, abl + n, size=count)
    b[np.arange(count), iy, ix] = 1.0
    return b


def random_complex(shape, seed: int) -> np.ndarray:
    """i.i.d. complex normal array (real and imaginary parts N(0,1))."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def smooth_plus_noise(count: int, N: int, seed: int, ell: float = 4.0,
                      noise: float = 0.1) -> np.ndarray:
    """Random training vectors x: a complex Gaussian random field (correlation
    length ell cells) plus `noise` times complex white noise, each sample
    scaled to unit RMS.  complex128 [count][N][N]."""
    rng = np.random.default_rng(seed)
    out = np.empty((count, N, N), dtype=np.complex128)
    for i in range(count):
        re = gaussian_filter(rng.standard_normal((N, N)), ell / np.sqrt(2.0), mode="wrap")
        im = gaussian_filter(rng.standard_normal((N, N)), ell / np.sqrt(2.0), mode="wrap")
        f = re + 1j * im
        f /= np.sqrt(np.mean(np.abs(f) ** 2))
        f += noise * (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
        out[i] = f
    return out


def iteration_counts(count: int, seed: int, lo: int = 2, hi: int = 20) -> np.ndarray:
    """Per-sample FGMRES iteration counts drawn uniformly from {lo..hi}."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=count).astype(np.int32)


def kaiming_uniform(shape, fan_in: int, rng: np.random.Generator) -> np.ndarray:
    """PyTorch's default conv initialisation: U(-b, b) with b = 1/sqrt(fan_in)."""
    b = 1.0 / np.sqrt(fan_in)
    return rng.uniform(-b, b, size=shape)


def random_params(spec, seed: int, bn_jitter: float = 0.0) -> dict:
    """Draw parameters for a list of (name, shape, fan_in, kind) entries.

    kind 'w'   : Kaiming-uniform weights (fan_in given)
    kind 'bn_g': ones (+ optional uniform jitter)
    kind 'bn_b': zeros (+ optional uniform jitter)
    kind 'bias': U(-1/sqrt(fan_in), 1/sqrt(fan_in))
    kind 'fixed': values supplied in the spec entry's 5th field (copied)
    """
    rng = np.random.default_rng(seed)
    out = {}
    for ent in spec:
        name, shape, fan_in, kind = ent[:4]
        if kind in ("w", "bias"):
            out[name] = kaiming_uniform(shape, fan_in, rng)
        elif kind == "bn_g":
            out[name] = np.ones(shape) + bn_jitter * rng.uniform(-1, 1, size=shape)
        elif kind == "bn_b":
            out[name] = np.zeros(shape) + bn_jitter * rng.uniform(-1, 1, size=shape)
        elif kind == "fixed":
            out[name] = np.array(ent[4], dtype=np.float64).reshape(shape).copy()
        else:
            raise ValueError(kind)
    return out
