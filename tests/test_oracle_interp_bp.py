"""Pins of the oracle's pixel-driven interpolating backprojector against independent facts: the
oracle's own rays (built in C) pass through the detector coordinate the backprojector assigns them,
the ray density |grad t| is the derivative of that coordinate, a constant sinogram gives V / ds for
parallel beams, and on smooth data the backprojector approximates the exact adjoint (pinned
separately) with the same scale."""

from __future__ import annotations

import math

import numpy as np
import pytest

import oracle as O
from synth import gaussian_blob, uniform_angles

GEOMS = {
    "parallel": dict(kind="parallel", n=40, angles=uniform_angles(12, math.pi) + 0.05, det_count=61,
                     det_spacing=0.8),
    "fan": dict(kind="fan", n=40, angles=uniform_angles(12, 2 * math.pi) + 0.05, det_count=90,
                source_distance=90.0, det_distance=60.0),
}


def _t_at(g, v, x, y):
    """Detector coordinate of an arbitrary point (x, y) (pixel-centred coordinates): the same
    definition as detector_coordinate, evaluated at any point rather than on the pixel grid."""
    th = float(g.angles[v])
    n = np.array([np.cos(th), np.sin(th)])
    u = np.array([-np.sin(th), np.cos(th)])
    cn = x * n[0] + y * n[1]
    if g.kind == "fan":
        s = (g.source_distance + g.det_distance) * cn / (x * u[0] + y * u[1] + g.source_distance)
    else:
        s = cn
    return s / g.det_spacing + (g.det_count - 1) / 2.0


@pytest.mark.parametrize("kind", list(GEOMS))
def test_rays_pass_through_their_detector_coordinate(kind):
    g = O.Geometry.from_args(GEOMS[kind])
    for v in range(0, g.n_angles, 3):
        for d in (0, 17, g.det_count // 2, g.det_count - 1):
            m, u = O.ray(g, v, d)                   # built by the C oracle
            for lam in (-7.0, 0.0, 5.5):
                p = m + lam * u
                assert _t_at(g, v, p[0], p[1]) == pytest.approx(d, abs=1e-9)
    # the grid function agrees with the point formula at the pixel centres
    t, _ = O.detector_coordinate(g, 4)
    c0 = (g.n - 1) / 2.0
    assert t[5, 9] == pytest.approx(_t_at(g, 4, 9 - c0, 5 - c0), abs=1e-12)


@pytest.mark.parametrize("kind", list(GEOMS))
def test_ray_density_is_the_gradient_of_the_detector_coordinate(kind):
    g = O.Geometry.from_args(GEOMS[kind])
    c0 = (g.n - 1) / 2.0
    _, w = O.detector_coordinate(g, 7)
    eps = 1e-5
    for (i, j) in ((0, 0), (13, 29), (39, 5)):
        x, y = j - c0, i - c0
        gx = (_t_at(g, 7, x + eps, y) - _t_at(g, 7, x - eps, y)) / (2 * eps)
        gy = (_t_at(g, 7, x, y + eps) - _t_at(g, 7, x, y - eps)) / (2 * eps)
        assert w[i, j] == pytest.approx(math.hypot(gx, gy), rel=1e-7)


def test_constant_sinogram_parallel_closed_form():
    g = O.Geometry("parallel", 20, uniform_angles(9, math.pi), 40, 0.9)
    b = O.backproject_interpolating(g, np.ones(g.sino_shape))
    # every pixel centre projects inside the detector: V views of weight 1 / ds
    assert np.allclose(b, 9 / 0.9, rtol=1e-13)


@pytest.mark.parametrize("kind", list(GEOMS))
def test_approximates_the_exact_adjoint_on_smooth_data(kind):
    g = O.Geometry.from_args(GEOMS[kind])
    y = O.forward(g, gaussian_blob(g.n, 3.0, -2.0, 6.0))
    bi = O.backproject_interpolating(g, y)
    ba = O.adjoint(g, y)
    # measured 1.8 % (parallel) and 0.7 % (fan); sums agree to 1.5e-4
    assert np.linalg.norm(bi - ba) <= 0.025 * np.linalg.norm(ba)
    assert bi.sum() / ba.sum() == pytest.approx(1.0, abs=1e-3)
