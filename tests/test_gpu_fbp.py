"""Filtered backprojection on the GPU (Section 3.1.3) against the FP64 oracle: the filter of every
window in every storage type, the reconstruction, the filter's autograd (it is symmetric), and the
paper's FBP setting (512^2, 512 views in [0, pi), ceil(512 sqrt 2) = 725 detectors)."""

from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle as O
from gpu_cases import TOL_F32, phantoms, rel_l2, to_dev, to_np, within_16
from paper_2009_14788_gb300 import Geometry, Radon, backward_raw, filter_sinogram
from synth import ellipse_phantom, uniform_angles

pytestmark = pytest.mark.gpu

CASES = {
    "parallel_64": dict(kind="parallel", n=64, angles=uniform_angles(96, math.pi), det_count=91),
    "parallel_ragged": dict(kind="parallel", n=37, angles=uniform_angles(50, math.pi) + 0.02, det_count=53,
                            det_spacing=0.9),
    "one_bin": dict(kind="parallel", n=8, angles=uniform_angles(3, math.pi), det_count=1),
    "fan_47": dict(kind="fan", n=47, angles=uniform_angles(30, 2 * math.pi), det_count=70, source_distance=120.0,
                   det_distance=60.0),
}


def _geoms(args):
    a = dict(args)
    kind = a.pop("kind")
    return Geometry(kind, **a), O.Geometry.from_args(args)


@pytest.mark.parametrize("name", O.FILTERS)
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16], ids=["f32", "f16", "bf16"])
def test_filter_matches_oracle(case, name, dtype):
    g, og = _geoms(CASES[case])
    y = np.random.default_rng(7).normal(size=(3,) + og.sino_shape)
    yd = to_dev(y, dtype)
    got = to_np(filter_sinogram(g, yd, name))
    ref = O.filter_sinogram(og, to_np(yd), name)
    if dtype == torch.float32:
        assert rel_l2(got, ref) <= TOL_F32
    else:
        assert within_16(got, ref, dtype), rel_l2(got, ref)


@pytest.mark.parametrize("name", ["ram-lak", "hann"])
def test_fbp_matches_oracle(name):
    g, og = _geoms(CASES["parallel_64"])
    x = phantoms(g.n, 2, seed=21)
    y = O.forward(og, x)
    rec = to_np(Radon(g.n, CASES["parallel_64"]["angles"], det_count=91).fbp(to_dev(y), name))
    ref = O.fbp(og, y.astype(np.float32).astype(np.float64), name)
    assert rel_l2(rec, ref) <= TOL_F32


def test_filter_gradient_is_the_filter():
    """The filter kernel is even, so the operator is symmetric: its gradient applies it again."""
    g, og = _geoms(CASES["parallel_ragged"])
    r = Radon(g.n, CASES["parallel_ragged"]["angles"], det_count=53, det_spacing=0.9)
    y = to_dev(np.random.default_rng(1).normal(size=(2,) + og.sino_shape)).requires_grad_(True)
    w = np.random.default_rng(2).normal(size=(2,) + og.sino_shape)
    (r.filter_sinogram(y, "shepp-logan") * to_dev(w)).sum().backward()
    assert rel_l2(to_np(y.grad), O.filter_sinogram(og, w, "shepp-logan")) <= TOL_F32


def test_filter_refuses_overlap_and_keeps_input():
    g, og = _geoms(CASES["parallel_64"])
    y = to_dev(np.random.default_rng(4).normal(size=(1,) + og.sino_shape))
    keep = y.clone()
    from paper_2009_14788_gb300._lib import RadonError
    with pytest.raises(RadonError):
        filter_sinogram(g, y, "ram-lak", out=y)
    assert torch.equal(y, keep)


def test_paper_fbp_setting_full_size():
    """512^2 phantom, 512 views in [0, pi), 725 detectors of spacing 1 (the paper's FBP setting):
    the GPU reconstruction equals the oracle's, and reconstructs the phantom."""
    n = 512
    angles = uniform_angles(512, math.pi)
    D = int(math.ceil(math.sqrt(2) * n))
    g = Geometry("parallel", n, angles, det_count=D, det_spacing=1.0)
    og = O.Geometry("parallel", n, angles, D, 1.0)
    x = ellipse_phantom(n, 10, 4242)
    y = O.forward(og, x)
    q = filter_sinogram(g, to_dev(y[None]), "ram-lak")
    rec = to_np(backward_raw(g, q))[0]
    ref = O.fbp(og, y.astype(np.float32).astype(np.float64), "ram-lak")
    assert rel_l2(rec, ref) <= TOL_F32
    # piecewise-constant phantom: the edges dominate the error (the oracle's own FBP: 2.51 %)
    assert rel_l2(rec, x) <= 0.03
