"""Seeded ellipse / Gaussian phantoms and angle sets.

Pixel convention (shared by every consumer): image ``x[i, j]`` has row ``i`` and
column ``j``; its centre sits at ``(j - (N-1)/2, i - (N-1)/2)``.  The paper's
experiments use the Shepp-Logan phantom (Section 3.1); these seeded random
ellipse phantoms stand in for it with the same piecewise-constant structure.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class EllipseSpec:
    x0: float       # centre, pixel units, image-centred
    y0: float
    a: float        # semi-axis along the rotated x axis
    b: float        # semi-axis along the rotated y axis
    phi: float      # rotation, radians
    rho: float      # additive intensity


def random_ellipses(n: int, count: int, seed: int, axes: tuple[float, float] | None = None) -> list[EllipseSpec]:
    """``count`` ellipses with semi-axes ~ U[axes], intensity ~ U[0,1], rotation ~ U[0, pi).

    The centre is uniform in the disk that keeps the whole ellipse inside the
    image's inscribed circle (radius N/2).  Default axes scale with N:
    U[N/16, 0.3125 N] (for N = 64 this is U[4, 20]).
    """
    rng = np.random.default_rng(seed)
    lo, hi = axes if axes is not None else (n / 16.0, 0.3125 * n)
    out = []
    for _ in range(count):
        a = rng.uniform(lo, hi)
        b = rng.uniform(lo, hi)
        rho = rng.uniform(0.0, 1.0)
        phi = rng.uniform(0.0, np.pi)
        r_max = max(0.0, n / 2.0 - max(a, b))
        # uniform in a disk: sqrt of a uniform radius fraction
        r = r_max * np.sqrt(rng.uniform(0.0, 1.0))
        t = rng.uniform(0.0, 2.0 * np.pi)
        out.append(EllipseSpec(r * np.cos(t), r * np.sin(t), a, b, phi, rho))
    return out


def _pixel_grid(n: int, supersample: int):
    c = (n - 1) / 2.0
    if supersample == 1:
        offs = np.zeros(1)
    else:
        offs = (np.arange(supersample) + 0.5) / supersample - 0.5
    xs = (np.arange(n)[:, None] + offs[None, :]).reshape(-1) - c
    return xs  # sub-sample coordinates along one axis, length n*supersample


def rasterize_ellipses(ellipses: list[EllipseSpec], n: int, supersample: int = 1, dtype=np.float64) -> np.ndarray:
    """Point-sample the additive ellipses at pixel centres (or an s x s sub-grid, averaged)."""
    coords = _pixel_grid(n, supersample)
    X = coords[None, :]
    Y = coords[:, None]
    img = np.zeros((coords.size, coords.size), dtype=np.float64)
    for e in ellipses:
        c, s = np.cos(e.phi), np.sin(e.phi)
        dx = X - e.x0
        dy = Y - e.y0
        xr = c * dx + s * dy
        yr = -s * dx + c * dy
        img += e.rho * ((xr / e.a) ** 2 + (yr / e.b) ** 2 <= 1.0)
    if supersample > 1:
        img = img.reshape(n, supersample, n, supersample).mean(axis=(1, 3))
    return img.astype(dtype)


def ellipse_phantom(n: int, count: int, seed: int, axes=None, dtype=np.float64) -> np.ndarray:
    return rasterize_ellipses(random_ellipses(n, count, seed, axes), n, 1, dtype)


def gaussian_blob(n: int, x0: float, y0: float, sigma: float, amp: float = 1.0) -> np.ndarray:
    """Isotropic Gaussian ``amp * exp(-|p - c|^2 / (2 sigma^2))`` sampled at pixel centres."""
    coords = np.arange(n) - (n - 1) / 2.0
    X = coords[None, :]
    Y = coords[:, None]
    return amp * np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / (2.0 * sigma * sigma))


def uniform_angles(count: int, span: float) -> np.ndarray:
    """``count`` angles equally spaced in ``[0, span)`` (the paper's ``np.linspace(..., endpoint=False)``)."""
    return np.linspace(0.0, span, count, endpoint=False)
