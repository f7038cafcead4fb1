"""The pixel-driven interpolating backprojector on the GPU against the FP64 oracle (parallel and fan,
every storage type, ragged sizes, a detector of one bin) and its relation to the exact adjoint."""

from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as O
from gpu_cases import TOL_F32, make, rel_l2, to_dev, to_np, within_16
from paper_2009_14788_gb300 import backproject_interpolating, backward_raw
from synth import gaussian_blob

pytestmark = pytest.mark.gpu

IBP_CASES = ["parallel_n64_full", "fan_n512_sub", "parallel_ragged", "fan_ragged", "fan_steep", "one_ray",
             "one_pixel", "parallel_fine"]


@pytest.mark.parametrize("path", ["packed", "plain"])
@pytest.mark.parametrize("case", IBP_CASES)
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16], ids=["f32", "f16", "bf16"])
def test_interpolating_backprojection_matches_oracle(case, dtype, path):
    """Both forms: the packed TMA pipeline (with a workspace; shapes it refuses fall back) and the
    plain one-thread-per-pixel kernel."""
    g, og = make(case)
    y = np.random.default_rng(11).uniform(0.0, 1.0, (10,) + og.sino_shape)   # 10 images: two CTA groups
    yd = to_dev(y, dtype)
    got = to_np(backproject_interpolating(g, yd, workspace="auto" if path == "packed" else None))
    ref = O.backproject_interpolating(og, to_np(yd))
    if dtype == torch.float32:
        assert rel_l2(got, ref) <= TOL_F32, rel_l2(got, ref)
    else:
        assert within_16(got, ref, dtype), rel_l2(got, ref)


def test_interpolating_backprojection_approximates_the_adjoint():
    g, og = make("fan_n512_block")
    y = O.forward(og, gaussian_blob(g.n, 10.0, -30.0, 40.0))
    bi = to_np(backproject_interpolating(g, to_dev(y[None])))[0]
    ba = to_np(backward_raw(g, to_dev(y[None])))[0]
    assert np.linalg.norm(bi - ba) <= 0.03 * np.linalg.norm(ba)
