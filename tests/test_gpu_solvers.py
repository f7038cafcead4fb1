"""Conjugate-gradient solvers on the GPU against the FP64 oracle (Section 4.2; Hanke's CGNE): the
batched vector kernels, CGNE run on the device, CG on a regularised normal operator built from the
fused projections, and the degenerate starts.

Tolerance of the K-step recursions: CG in finite precision loses orthogonality on an ill-posed
system, so FP32 rounding grows quickly with K (an FP32 model of the oracle's recursion parts from
FP64 by 1e-7, 8e-6 and 8e-3 at K = 2, 5 and 10).  Early iterates are gated against the FP64 oracle,
later ones against that FP32 model; the reconstruction error against the truth is gated too."""

from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle as O
from gpu_cases import phantoms, rel_l2, to_dev, to_np
from paper_2009_14788_gb300 import Geometry, backward_fused, cg, cgne, forward_raw
from paper_2009_14788_gb300.solvers import _Vec
from synth import uniform_angles

pytestmark = pytest.mark.gpu

SMALL = dict(kind="parallel", n=64, angles=uniform_angles(30, math.pi), det_count=91)
FAN = dict(kind="fan", n=48, angles=uniform_angles(24, 2 * math.pi) + 0.1, det_count=80, source_distance=150.0,
           det_distance=90.0)
TOL_CG5 = 5e-5          # K = 5 FP32 steps against FP64 (measured 3.5e-6 .. 5.5e-6)
TOL_CG10_MODEL = 5e-4   # K = 10 against the FP32 model of the recursion (measured 2.5e-5 .. 6.7e-5)
# K = 10 against FP64 directly: an FP32 recursion (the model, exact projections) departs from FP64 by
# 8.4e-3 (parallel) and 1.1e-2 (fan) on these cases; the gate allows ~3x that departure.  FP64
# recursions with a planted mistake depart by 4.1e-2 .. 4.9e-2 (direction-update coefficient 10 %
# off), 9.0e-2 .. 9.2e-2 (step length 10 % short), 0.10 (no direction update) and 2.4 (step 10 % long)
TOL_CG10_FP64 = 3e-2


def _geoms(args):
    a = dict(args)
    kind = a.pop("kind")
    return Geometry(kind, **a), O.Geometry.from_args(args)


@pytest.mark.parametrize("batch", [1, 3, 40])
def test_batched_dot_and_axpby(batch):
    rng = np.random.default_rng(batch)
    a, b = rng.normal(size=(batch, 777)), rng.normal(size=(batch, 777))
    ad, bd = to_dev(a), to_dev(b)
    v = _Vec(batch, ad.device)
    out = torch.empty(batch, device="cuda")
    v.dot(ad, bd, out)
    ref = np.sum(to_np(ad) * to_np(bd), axis=1)
    assert np.allclose(to_np(out), ref, rtol=0, atol=2e-6 * np.sum(np.abs(a * b), axis=1).max())
    s = to_dev(rng.uniform(0.5, 2.0, batch))
    t = to_dev(rng.uniform(-1.0, 1.0, batch))
    y = bd.clone()
    v.axpby(ad, y, 0.5, alpha_dev=s, beta=2.0, beta_dev=t)
    ref = 0.5 * to_np(s)[:, None] * to_np(ad) + 2.0 * to_np(t)[:, None] * to_np(bd)
    assert np.allclose(to_np(y), ref, rtol=1e-6, atol=1e-6)
    den = to_dev(np.where(np.arange(batch) % 2 == 0, 0.0, 2.0))
    q = torch.empty(batch, device="cuda")
    v.divide(s, den, q)
    assert np.allclose(to_np(q), np.where(np.arange(batch) % 2 == 0, 0.0, to_np(s) / 2.0))


def _f32(a):
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def _dot(a, b):
    return _f32(np.sum(a.reshape(a.shape[0], -1) * b.reshape(b.shape[0], -1), axis=1))


def cgne_f32_model(og, x0, y, iterations):
    """The oracle's CGNE recursion with every vector and scalar rounded to FP32 after each step (the
    kernel's storage), projections exact: a model of what FP32 arithmetic does to the recursion."""
    x = _f32(x0)
    r = _f32(y - O.forward(og, x))
    s = _f32(O.adjoint(og, r))
    p = s.copy()
    gam = _dot(s, s)
    e = (slice(None), None, None)
    for _ in range(iterations):
        q = _f32(O.forward(og, p))
        a = _f32(gam / _dot(q, q))
        x = _f32(x + a[e] * p)
        r = _f32(r - a[e] * q)
        s = _f32(O.adjoint(og, r))
        gn = _dot(s, s)
        p = _f32(s + _f32(gn / gam)[e] * p)
        gam = gn
    return x


@pytest.mark.parametrize("args", [SMALL, FAN], ids=["parallel", "fan"])
def test_cgne_matches_oracle(args):
    """Early iterates against the FP64 oracle; later ones against the FP32 model of the recursion
    (CG in finite precision loses orthogonality on an ill-posed system and converges more slowly --
    the FP32 and FP64 recursions part by ~1e-2 at K = 10 -- while its reconstruction error stays)."""
    g, og = _geoms(args)
    x_true = phantoms(g.n, 3, seed=31)
    y = O.forward(og, x_true) + np.random.default_rng(31).normal(0.0, 0.01, (3,) + og.sino_shape)
    y32 = _f32(y)
    x0 = np.zeros((3, g.n, g.n))
    got5 = to_np(cgne(g, to_dev(x0), to_dev(y32), 5))
    e5 = rel_l2(got5, O.cgne(og, x0, y32, 5))
    got10 = to_np(cgne(g, to_dev(x0), to_dev(y32), 10))
    e10 = rel_l2(got10, cgne_f32_model(og, x0, y32, 10))
    ref10 = O.cgne(og, x0, y32, 10)
    print("CGNE: K=5 vs FP64 %.3g, K=10 vs FP32 model %.3g, K=10 vs FP64 %.3g" % (e5, e10, rel_l2(got10, ref10)))
    assert e5 <= TOL_CG5, e5
    assert e10 <= TOL_CG10_MODEL, e10
    assert rel_l2(got10, ref10) <= TOL_CG10_FP64, rel_l2(got10, ref10)
    # the reconstruction error against the truth is that of the exact recursion
    assert abs(rel_l2(got10, x_true) - rel_l2(ref10, x_true)) <= 0.02 * rel_l2(ref10, x_true)
    assert np.linalg.norm(O.forward(og, got10) - y) < 0.5 * np.linalg.norm(y)


def test_cgne_degenerate_starts():
    g, og = _geoms(SMALL)
    x0 = to_dev(phantoms(g.n, 2, seed=2))
    keep = x0.clone()
    y = forward_raw(g, x0)                          # consistent data from the start itself ...
    out0 = cgne(g, x0, y, 0)
    assert torch.equal(out0, x0) and out0.data_ptr() != x0.data_ptr()
    z = cgne(g, torch.zeros_like(x0), torch.zeros_like(y), 5)
    assert torch.equal(z, torch.zeros_like(z))      # zero data: every step length is zero, no NaN
    assert torch.equal(x0, keep)


def test_cg_on_regularised_normal_operator_matches_oracle():
    """CG for (A^T A + lambda I) x = A^T y; the operator runs as one forward and one fused adjoint."""
    g, og = _geoms(FAN)
    lam = 5.0
    x_true = phantoms(g.n, 2, seed=41)
    y = O.forward(og, x_true).astype(np.float32).astype(np.float64)
    b = O.adjoint(og, y)

    def op_gpu(x):
        return backward_fused(g, forward_raw(g, x), add=x, add_scale=lam)

    def op_ref(x):
        return O.adjoint(og, O.forward(og, x)) + lam * x

    got = to_np(cg(op_gpu, torch.zeros((2, g.n, g.n), device="cuda"), to_dev(b), 5))
    ref = O.cg(op_ref, np.zeros((2, g.n, g.n)), _f32(b), 5)
    print("CG: K=5 vs FP64 %.3g" % rel_l2(got, ref))
    assert rel_l2(got, ref) <= TOL_CG5, rel_l2(got, ref)
