"""Pins of the oracle's filtered backprojection (Section 3.1.3; filter construction of Kak & Slaney,
Chapter 3, Eq. 61) against what the mathematics fixes, independent of the oracle's own code path."""

from __future__ import annotations

import math

import numpy as np
import pytest

import oracle as O
from synth import gaussian_blob, uniform_angles


def test_ramp_response_is_the_ideal_ramp():
    """The DTFT of the band-limited ramp kernel is |f| on [-1/2, 1/2]; the length-P DFT of its
    truncation differs only by the discarded tail (sum over |m| > P/2 of 2 / (pi^2 m^2) < 4 / (pi^2 P))."""
    for D in (7, 91, 725):
        P = O.filter_length(D)
        assert P >= 2 * D - 1 and P & (P - 1) == 0
        H = O.frequency_filter("ram-lak", D)
        f = np.fft.fftfreq(P)
        tail = 4.0 / (np.pi ** 2 * P)
        assert np.max(np.abs(H - np.abs(f))) <= tail
        assert 0.0 < H[0] <= tail          # no zero at DC: the point of building the filter in space


def test_fft_route_equals_direct_convolution_with_the_spatial_kernel():
    """Zero padding to P >= 2D - 1 makes the circular convolution a linear one: filtering equals a
    direct sum over detectors with the Eq. 61 kernel, which pins padding, orientation and scale."""
    rng = np.random.default_rng(3)
    g = O.Geometry("parallel", 16, uniform_angles(5, math.pi), 23)
    y = rng.normal(size=(2,) + g.sino_shape)
    got = O.filter_sinogram(g, y, "ram-lak")
    d = np.arange(g.det_count)
    K = O.ramp_kernel(d[:, None] - d[None, :])          # [out, in]
    ref = (np.pi / g.n_angles) * np.einsum("oi,bvi->bvo", K, y)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_windows_shape_the_ramp():
    """Each window is 1 at DC and only attenuates; at the band edge cosine and Hann vanish, Hamming
    keeps 0.08, Shepp-Logan 2/pi, Ram-Lak all of it."""
    edge = {"ram-lak": 1.0, "shepp-logan": 2 / np.pi, "cosine": 0.0, "hamming": 0.08, "hann": 0.0}
    f = np.linspace(-0.5, 0.5, 201)
    for name in O.FILTERS:
        w = O.window(name, f)
        assert w[100] == pytest.approx(1.0)
        assert np.all(w <= 1.0 + 1e-15) and np.all(w >= -1e-15)
        assert w[0] == pytest.approx(edge[name], abs=1e-12) and w[-1] == pytest.approx(edge[name], abs=1e-12)
        assert np.all(np.diff(w[100:]) <= 1e-15)       # non-increasing away from DC
    with pytest.raises(ValueError):
        O.window("lanczos", f)


@pytest.mark.parametrize("name", O.FILTERS)
def test_fbp_reconstructs_a_smooth_phantom(name):
    """FBP of the projections of a smooth blob, dense views in [0, pi), detectors covering the
    image diagonal: the reconstruction matches the blob (smoother windows lose a little contrast)."""
    n = 64
    x = gaussian_blob(n, 4.0, -6.0, 7.0) + 0.5 * gaussian_blob(n, -10.0, 8.0, 4.0)
    g = O.Geometry("parallel", n, uniform_angles(180, math.pi), int(math.ceil(n * math.sqrt(2))))
    rec = O.fbp(g, O.forward(g, x), name)
    err = np.linalg.norm(rec - x) / np.linalg.norm(x)
    # measured 1.10 / 1.19 / 1.39 / 1.68 / 1.74 %
    assert err <= {"ram-lak": 0.015, "shepp-logan": 0.015, "cosine": 0.02, "hamming": 0.025, "hann": 0.025}[name], err
    # the scale pi / V: a factor-two or missing-pi mistake moves the mean by 100 % or more (measured 4e-5)
    assert abs(rec.sum() / x.sum() - 1.0) <= 1e-3


def test_smoothing_windows_reduce_noise_gain():
    """On white noise the reconstruction's energy falls from Ram-Lak to the windowed filters, in the
    order of the windows' high-frequency energy (Hann < Hamming < cosine < Shepp-Logan < Ram-Lak)."""
    g = O.Geometry("parallel", 32, uniform_angles(48, math.pi), 46)
    noise = np.random.default_rng(9).normal(size=g.sino_shape)
    e = {name: float(np.linalg.norm(O.fbp(g, noise, name))) for name in O.FILTERS}
    assert e["hann"] < e["hamming"] < e["cosine"] < e["shepp-logan"] < e["ram-lak"]
