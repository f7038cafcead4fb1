"""Landweber iteration on the GPU (Section 4.2) against the FP64 oracle: the fused residual and
update epilogues, the inner product and scaled add, the power-method step size, the iterates, and
the reverse-mode gradients w.r.t. y and alpha through all iterations (per-iteration checkpoints).

Tolerances.  One FP32 projection is gated at rel-L2 1e-5.  A K-step chain composes 2K projections
through a non-expansive map (alpha <= 1 / lambda_max, so I - alpha A^T A has norm <= 1): the
relative error of the iterate stays within the sum of the per-step errors, 2K * 1e-6 (measured
single-op errors sit near 1e-7 .. 1e-6), so the FP32 chain gate is 1e-5 * ceil(2K / 10) = 2e-5
at K = 10.  With 16-bit storage every stored iterate and residual is rounded once more, an
independent relative error of RMS <= 2^-9 per element; the chain adds at most 2K + 1 such
roundings, each damped by the non-expansive map, so the 16-bit chain gate is
2e-3 * sqrt(2K + 1) (9.2e-3 at K = 10).
"""

from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle as O
from gpu_cases import TOL_16, TOL_F32, phantoms, rel_l2, to_dev, to_np
from paper_2009_14788_gb300 import (Geometry, Landweber, axpby, backward_fused, dot, forward_fused, forward_raw,
                                    power_iteration)
from synth import WORKLOADS, power_start, uniform_angles, workload_geometry_args, workload_images, workload_noise

pytestmark = pytest.mark.gpu

K = 10


def chain_tol_f32(k: int) -> float:
    return TOL_F32 * math.ceil(2 * k / 10)


def chain_tol_16(k: int) -> float:
    return TOL_16 * math.sqrt(2 * k + 1)


SMALL = dict(kind="parallel", n=64, angles=uniform_angles(30, math.pi), det_count=91, det_spacing=1.0)
SMALL_FAN = dict(kind="fan", n=48, angles=uniform_angles(24, 2 * math.pi) + 0.1, det_count=80,
                 source_distance=150.0, det_distance=90.0)


def _geoms(args):
    a = dict(args)
    kind = a.pop("kind")
    return Geometry(kind, **a), O.Geometry.from_args(args)


def _rounded(a: np.ndarray, dtype) -> np.ndarray:
    """The values a tensor of ``dtype`` holds after the host array is copied in."""
    return to_np(to_dev(a, dtype))


@pytest.mark.parametrize("args", [SMALL, SMALL_FAN], ids=["parallel", "fan"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16], ids=["f32", "bf16", "f16"])
def test_fused_residual_keeps_its_own_precision(args, dtype):
    """r = A x - y in one kernel, rounded once: the storage rounding is relative to |r|.

    The FP32 accumulation of A x carries the projection's own error (gate 1e-5 of |A x|); the
    16-bit store adds at most one rounding of r itself (gate 2e-3 of |r|).  Rounding A x to 16 bits
    before subtracting would instead add an error of order 2e-3 |A x|, far above both."""
    g, og = _geoms(args)
    x_true = phantoms(g.n, 3, seed=11)
    x = x_true * 0.98 + 0.01                                     # a nearby iterate: r is small against A x
    y = O.forward(og, x_true)
    xd, yd = to_dev(x, dtype), to_dev(y, dtype)
    ax = O.forward(og, _rounded(x, dtype))
    ref = ax - _rounded(y, dtype)
    got = forward_fused(g, xd, add=yd, add_scale=-1.0)
    err = np.linalg.norm(to_np(got) - ref)
    bound = TOL_F32 * np.linalg.norm(ax) + (0.0 if dtype == torch.float32 else TOL_16 * np.linalg.norm(ref))
    assert err <= bound
    assert np.linalg.norm(ref) < 0.2 * np.linalg.norm(ax)        # the case is a cancelling one
    if dtype != torch.float32:
        assert err < 0.25 * TOL_16 * np.linalg.norm(ax)          # far below what a rounded A x would give


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
@pytest.mark.parametrize("algo_ws", ["packed", "plain"])
def test_fused_update_in_place(dtype, algo_ws):
    """x' = x - alpha A^T r with alpha on the device, written over x (the addend is the output)."""
    g, og = _geoms(SMALL_FAN)
    x = phantoms(g.n, 5, seed=3)
    r = np.random.default_rng(4).normal(0.0, 1.0, (5,) + og.sino_shape)
    alpha = 3.7e-3
    xd, rd = to_dev(x, dtype), to_dev(r, dtype)
    ad = torch.tensor([alpha], dtype=torch.float32, device="cuda")
    ref = _rounded(x, dtype) - alpha * O.adjoint(og, _rounded(r, dtype))
    kw = dict(workspace=None) if algo_ws == "plain" else {}
    out = backward_fused(g, rd, op_scale=-1.0, op_scale_dev=ad, add=xd, add_scale=1.0, out=xd, **kw)
    assert out.data_ptr() == xd.data_ptr()
    tol = TOL_F32 if dtype == torch.float32 else TOL_16
    assert rel_l2(to_np(xd), ref) <= tol


def test_identity_epilogue_is_bit_exact():
    g, _ = _geoms(SMALL)
    x = to_dev(phantoms(g.n, 2, seed=5))
    a = forward_raw(g, x)
    b = forward_fused(g, x)
    assert torch.equal(a, b)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16], ids=["f32", "f16", "bf16"])
@pytest.mark.parametrize("count", [1, 1000, 777_777])
def test_dot_and_axpby(dtype, count):
    rng = np.random.default_rng(count)
    a, b = rng.normal(size=count), rng.normal(size=count)
    ad, bd = to_dev(a, dtype), to_dev(b, dtype)
    ar, br = to_np(ad), to_np(bd)
    res = dot(ad, bd, scale=-2.0)
    ref = -2.0 * float(np.dot(ar, br))
    # FP32 products summed in FP32 per thread (a few dozen terms) and FP64 beyond
    assert abs(float(res.item()) - ref) <= 1e-6 * float(np.dot(np.abs(ar), np.abs(br))) * 2 + 1e-30
    dot(ad, bd, result=res, scale=1.0, accumulate=True)
    assert abs(float(res.item()) - (ref + float(np.dot(ar, br)))) <= 4e-6 * float(np.dot(np.abs(ar), np.abs(br)))
    # deterministic: the same call gives the same bits
    assert torch.equal(dot(ad, bd), dot(ad, bd))
    y = torch.full((count,), float("nan"), dtype=torch.float32, device="cuda")
    axpby(ad, y, 0.5, beta=0.0)                                  # beta = 0 never reads y (NaN here)
    assert np.allclose(to_np(y), 0.5 * ar, rtol=1e-7, atol=0)
    s = torch.tensor([4.0], device="cuda")
    axpby(bd, y, 0.25, alpha_dev=s, beta=2.0)                    # y = 1 * b + 2 * (0.5 a)
    assert np.allclose(to_np(y), br + ar, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("args", [SMALL, SMALL_FAN], ids=["parallel", "fan"])
def test_power_iteration_matches_oracle(args):
    g, og = _geoms(args)
    seed = 20
    lam_ref = O.power_iteration(og, 20, seed)
    v0 = to_dev(power_start(g.n, seed))
    lam, alpha = power_iteration(g, v0, 20)
    assert abs(lam.item() - lam_ref) <= TOL_F32 * lam_ref
    assert abs(alpha.item() - 1.0 / lam_ref) <= TOL_F32 / lam_ref
    # the estimate approaches the largest eigenvalue of A^T A from below (dense matrix, small case)
    if g.n <= 48:
        A = O.dense_matrix(og)
        top = float(np.linalg.eigvalsh(A.T @ A)[-1])
        assert lam_ref <= top * (1 + 1e-12) and lam_ref > 0.9 * top


def _landweber_case(args, batch, dtype, seed=9):
    g, og = _geoms(args)
    x_true = phantoms(g.n, batch, seed=seed)
    y = O.forward(og, x_true) + np.random.default_rng(seed).normal(0.0, 0.01, (batch,) + og.sino_shape)
    lam = O.power_iteration(og, 20, seed)
    return g, og, x_true, y, 1.0 / lam


@pytest.mark.parametrize("args", [SMALL, SMALL_FAN], ids=["parallel", "fan"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
def test_landweber_iterates_match_oracle(args, dtype):
    g, og, x_true, y, alpha = _landweber_case(args, 3, dtype)
    yd = to_dev(y, dtype)
    x0 = torch.zeros((3, g.n, g.n), dtype=dtype, device="cuda")
    xk = Landweber(g).run(x0, yd, alpha, K)
    ref = O.landweber(og, np.zeros((3, g.n, g.n)), _rounded(y, dtype), float(np.float32(alpha)), K)
    tol = chain_tol_f32(K) if dtype == torch.float32 else chain_tol_16(K)
    assert rel_l2(to_np(xk), ref) <= tol
    # the iteration reduces the data misfit
    assert np.linalg.norm(O.forward(og, to_np(xk)) - y) < 0.9 * np.linalg.norm(y)


@pytest.mark.parametrize("args", [SMALL, SMALL_FAN], ids=["parallel", "fan"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
def test_landweber_gradients_match_oracle(args, dtype):
    """dL/dy and dL/dalpha of L = |x_K - x_true|^2 against the oracle's reverse mode."""
    g, og, x_true, y, alpha = _landweber_case(args, 2, dtype, seed=13)
    alpha = float(np.float32(alpha))
    yd = to_dev(y, dtype).requires_grad_(True)
    ad = torch.tensor([alpha], dtype=torch.float32, device="cuda", requires_grad=True)
    x0 = torch.zeros((2, g.n, g.n), dtype=dtype, device="cuda")
    xk = Landweber(g).run(x0, yd, ad, K)
    xt = to_dev(x_true, torch.float32)
    loss = ((xk.float() - xt) ** 2).sum()
    loss.backward()
    loss_ref, dy_ref, da_ref = O.landweber_grads(og, np.zeros((2, g.n, g.n)), _rounded(y, dtype), alpha, K,
                                                 to_np(xt))
    tol = chain_tol_f32(2 * K) if dtype == torch.float32 else chain_tol_16(2 * K)
    assert abs(loss.item() - loss_ref) <= tol * loss_ref
    assert rel_l2(to_np(yd.grad), dy_ref) <= tol
    assert abs(ad.grad.item() - da_ref) <= tol * abs(da_ref)


def test_landweber_gradient_x0_and_zero_iterations():
    g, og, x_true, y, alpha = _landweber_case(SMALL, 1, torch.float32)
    yd = to_dev(y)
    x0 = to_dev(x_true * 0.5).requires_grad_(True)
    xk = Landweber(g).run(x0, yd, alpha, 3)
    w = np.random.default_rng(1).normal(size=x_true.shape)
    (xk * to_dev(w)).sum().backward()
    # dL/dx0 = (I - alpha A^T A)^3 w
    ref = w.copy()
    for _ in range(3):
        ref = ref - float(np.float32(alpha)) * O.adjoint(og, O.forward(og, ref))
    assert rel_l2(to_np(x0.grad), ref) <= chain_tol_f32(6)
    x1 = to_dev(x_true).requires_grad_(True)
    out = Landweber(g).run(x1, yd, alpha, 0)
    assert out.data_ptr() != x1.data_ptr() and torch.equal(out, x1)
    out.sum().backward()
    assert torch.equal(x1.grad, torch.ones_like(x1))


def test_landweber_full_size_bf16_two_images():
    """The 8 x 512^2, 60-view, 725-detector bf16 workload, first two images, against the oracle."""
    w = WORKLOADS["landweber_b8_n512_v60_d725"]
    args = workload_geometry_args(w)
    g, og = _geoms(args)
    x_true = workload_images(w, [0, 1])
    y = O.forward(og, x_true) + workload_noise(w, (w.batch,) + og.sino_shape)[:2]
    v0 = to_dev(power_start(g.n, 2000 * w.number))
    lam, alpha = power_iteration(g, v0, w.extra["power_iterations"])
    lam_ref = O.power_iteration(og, w.extra["power_iterations"], 2000 * w.number)
    assert abs(lam.item() - lam_ref) <= TOL_F32 * lam_ref
    yd = to_dev(y, torch.bfloat16)
    x0 = torch.zeros((2, g.n, g.n), dtype=torch.bfloat16, device="cuda")
    xk = Landweber(g).run(x0, yd, alpha, w.extra["iterations"])
    ref = O.landweber(og, np.zeros((2, g.n, g.n)), _rounded(y, torch.bfloat16), float(alpha.item()),
                      w.extra["iterations"])
    assert rel_l2(to_np(xk), ref) <= chain_tol_16(w.extra["iterations"])
