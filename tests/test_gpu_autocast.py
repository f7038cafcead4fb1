"""Autocast (the paper's transparent half precision, Section 2): under torch.autocast the Radon
operators take FP32 tensors, run their 16-bit storage paths, and return gradients in FP32."""

from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle as O
from gpu_cases import TOL_16, phantoms, rel_l2, to_dev, to_np
from paper_2009_14788_gb300 import Radon, RadonFanbeam
from synth import uniform_angles

pytestmark = pytest.mark.gpu


def _radons():
    ang = uniform_angles(40, math.pi)
    fang = uniform_angles(36, 2 * math.pi)
    return [(Radon(64, ang, det_count=91), O.Geometry("parallel", 64, ang, 91)),
            (RadonFanbeam(64, fang, 150.0, det_distance=90.0, det_count=100),
             O.Geometry("fan", 64, fang, 100, None, 1.0, source_distance=150.0, det_distance=90.0))]


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16], ids=["f16", "bf16"])
@pytest.mark.parametrize("which", [0, 1], ids=["parallel", "fan"])
def test_autocast_runs_the_16bit_paths_and_returns_fp32_gradients(dtype, which):
    radon, og = _radons()[which]
    x = phantoms(64, 2, seed=3)
    xd = to_dev(x).requires_grad_(True)
    with torch.autocast("cuda", dtype=dtype):
        y = radon.forward(xd)
        b = radon.backprojection(y)
    assert y.dtype == dtype and b.dtype == dtype
    xr = to_np(to_dev(x, dtype))                     # the values the 16-bit path sees
    assert rel_l2(to_np(y), O.forward(og, xr)) <= TOL_16
    b.float().sum().backward()
    assert xd.grad.dtype == torch.float32
    # d/dx sum(A^T A x) = A^T A 1, through both operators' 16-bit paths
    ref = O.adjoint(og, O.forward(og, np.ones((2, 64, 64))))
    assert rel_l2(to_np(xd.grad), ref) <= 3 * TOL_16


def test_without_autocast_fp32_stays_fp32():
    radon, _ = _radons()[0]
    y = radon.forward(to_dev(phantoms(64, 1)))
    assert y.dtype == torch.float32
    with torch.autocast("cuda", dtype=torch.float16):
        y16 = radon.forward(to_dev(phantoms(64, 1), torch.float16))   # 16-bit inputs pass as they are
    assert y16.dtype == torch.float16
