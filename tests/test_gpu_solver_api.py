"""The solver interface the way the paper's reconstruction examples call it (Sections 4.2, 4.3): the
Landweber step from the image size and the device, ``run`` with ``iterations=``, ``cgne`` / ``cg``
with ``max_iter=``, ``cg`` on one image as one problem, and FBP, Landweber and CGNE reconstructing a
phantom.  Values against the FP64 oracle (dense eigenvalues, the oracle's iterations)."""

from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle as O
from gpu_cases import rel_l2, to_dev, to_np
from paper_2009_14788_gb300 import Landweber, Radon, cgne
from paper_2009_14788_gb300.solvers import cg
from synth import ellipse_phantom, uniform_angles

pytestmark = pytest.mark.gpu

TOL_CHAIN10 = 2e-5   # FP32 Landweber chain of 10 iterations (20 projections)
TOL_CG5 = 5e-5       # FP32 CG / CGNE after 5 iterations against FP64


def _setup(n=32, views=24):
    angles = uniform_angles(views, math.pi)
    det = int(math.ceil(n * math.sqrt(2.0)))
    radon = Radon(n, angles, det_count=det)
    og = O.Geometry.from_args(dict(kind="parallel", n=n, angles=angles, det_count=det))
    return radon, og, ellipse_phantom(n, 5, 21)


def test_estimate_alpha_takes_the_image_size_and_device():
    radon, og, _ = _setup(n=8, views=6)
    lw = Landweber(radon)
    alpha = lw.estimate_alpha(8, "cuda", n_iter=300)
    A = O.dense_matrix(og)
    lam = float(np.linalg.eigvalsh(A.T @ A).max())
    assert abs(float(alpha) * lam - 1.0) <= 1e-4
    alpha2, lam2 = lw.power(300)
    assert torch.equal(alpha, alpha2) and abs(float(lam2) / lam - 1.0) <= 1e-4
    with pytest.raises(ValueError):
        lw.estimate_alpha(9, "cuda")


def test_landweber_run_with_the_iterations_keyword():
    radon, og, x = _setup()
    y = O.forward(og, x[None]).astype(np.float32).astype(np.float64)   # inputs from the oracle
    alpha = 0.95 / O.power_iteration(og, 50, seed=1)
    rec = Landweber(radon).run(torch.zeros((1, 32, 32), device="cuda"), to_dev(y), alpha, iterations=10)
    ref = O.landweber(og, np.zeros((1, 32, 32)), y, alpha, 10)
    assert rel_l2(to_np(rec), ref) <= TOL_CHAIN10


def test_cgne_takes_max_iter():
    radon, og, x = _setup()
    y_np = O.forward(og, x[None]).astype(np.float32).astype(np.float64)
    y = to_dev(y_np)
    guess = torch.zeros((1, 32, 32), device="cuda")
    a = cgne(radon, guess, y, max_iter=5)
    assert torch.equal(a, cgne(radon, guess, y, 5)) and torch.equal(a, cgne(radon, guess, y, iterations=5))
    with pytest.raises(ValueError):
        cgne(radon, guess, y)
    with pytest.raises(ValueError):
        cgne(radon, guess, y, 5, iterations=5)
    assert rel_l2(to_np(a), O.cgne(og, np.zeros((1, 32, 32)), y_np, 5)) <= TOL_CG5


def test_cg_on_one_image_is_one_problem():
    """A two-dimensional start is one problem: the same bits as the batch of one."""
    radon, og, x = _setup()
    lam = 3.0
    b_np = O.adjoint(og, O.forward(og, x[None]))[0].astype(np.float32).astype(np.float64)
    b = to_dev(b_np)

    def op(v):
        return radon.backprojection(radon.forward(v)) + lam * v

    one = cg(op, torch.zeros_like(b), b, max_iter=5)
    assert one.shape == b.shape
    batch = cg(op, torch.zeros_like(b)[None], b[None], max_iter=5)[0]
    assert torch.equal(one, batch)
    ref = O.cg(lambda v: O.adjoint(og, O.forward(og, v)) + lam * v, np.zeros((1, 32, 32)), b_np[None], 5)[0]
    assert rel_l2(to_np(one), ref) <= TOL_CG5


def test_reconstructions_approach_the_phantom():
    """FBP, Landweber and CGNE from noiseless data: each ends closer to the phantom than the zero
    image, and the iterative ones improve with iterations."""
    n = 64
    angles = uniform_angles(96, math.pi)
    radon = Radon(n, angles, det_count=int(math.ceil(n * math.sqrt(2.0))))
    x = to_dev(ellipse_phantom(n, 5, 4)[None])
    y = radon.forward(x)

    def mse(r):
        return float(((r - x) ** 2).mean())

    base = mse(torch.zeros_like(x))
    assert mse(radon.fbp(y)) < 0.2 * base
    lw = Landweber(radon)
    alpha = lw.estimate_alpha(n, "cuda") * 0.95
    guess = torch.zeros_like(x)
    lw10, lw40 = lw.run(guess, y, alpha, iterations=10), lw.run(guess, y, alpha, iterations=40)
    assert mse(lw40) < mse(lw10) < base
    cg5, cg20 = cgne(radon, guess, y, max_iter=5), cgne(radon, guess, y, max_iter=20)
    assert mse(cg20) < mse(cg5) < base
