"""Batch-1 calls: under RADON_ALGO_AUTO with no tile parameters one image runs the single-image
kernels (the uneven-batch plan's per-image forward and adjoint, Section 4.1, launched without a
plan) instead of a batch-interleaved group it would fill to one slot.  Checked against the FP64
oracle on every shared geometry case in FP32 (rel-L2 1e-5) and 16-bit storage (2e-3, one storage
ulp for tiny outputs); bit for bit against a one-item plan with the same tile shape (the same
kernels); with fused epilogues; against the batched and workspace-free paths; and from a CUDA graph."""

from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as O
from gpu_cases import CASES, TOL_F32, make, phantoms, rel_l2, to_dev, to_np, within_16
from paper_2009_14788_gb300 import BatchPlan, _lib as L, backward_fused, backward_raw, forward_fused, forward_raw

pytestmark = pytest.mark.gpu

DTYPES = [torch.float32, torch.float16, torch.bfloat16]
DT_IDS = ["f32", "f16", "bf16"]


def _gate(got, ref, dtype):
    if dtype == torch.float32:
        return rel_l2(got, ref) <= TOL_F32
    return within_16(got, ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES, ids=DT_IDS)
@pytest.mark.parametrize("case", sorted(CASES))
def test_single_image_matches_oracle(case, dtype):
    g, og = make(case)
    x = to_dev(phantoms(g.n, 1, seed=11), dtype)
    y = forward_raw(g, x)
    ref = O.forward(og, to_np(x))
    assert _gate(to_np(y), ref, dtype), rel_l2(to_np(y), ref)
    ys = to_dev(np.random.default_rng(12).normal(size=(1,) + og.sino_shape), dtype)
    xb = backward_raw(g, ys)
    ref_b = O.adjoint(og, to_np(ys))
    assert _gate(to_np(xb), ref_b, dtype), rel_l2(to_np(xb), ref_b)


@pytest.mark.parametrize("direction", ["forward", "adjoint"])
@pytest.mark.parametrize("case", ["parallel_n64_full", "parallel_ragged", "fan_ragged", "fan_steep"])
def test_batch_one_is_the_plan_kernel(case, direction):
    """A batch-1 call equals, bit for bit, a one-item plan with the same tile shape."""
    g, og = make(case)
    if direction == "forward":
        inp = to_dev(phantoms(g.n, 1, seed=3))
        out_plan = torch.empty((1,) + g.sino_shape, device="cuda")
        plan = BatchPlan([(g, inp, out_plan)], "forward", autotune=False, forward_views=8, forward_lanes=4,
                         forward_kernel="gather")
        got = forward_raw(g, inp)
    else:
        inp = to_dev(np.random.default_rng(4).normal(size=(1,) + og.sino_shape))
        out_plan = torch.empty((1, g.n, g.n), device="cuda")
        plan = BatchPlan([(g, inp, out_plan)], "adjoint", autotune=False, adjoint_views=16)
        got = backward_raw(g, inp)
    plan.launch()
    torch.cuda.synchronize()
    assert torch.equal(got, out_plan)


@pytest.mark.parametrize("dtype", DTYPES, ids=DT_IDS)
def test_batch_one_fused_epilogues(dtype):
    """out = op_scale * s * P + add_scale * add at batch 1, against the oracle's P combined in FP64."""
    g, og = make("fan_ragged")
    x = to_dev(phantoms(g.n, 1, seed=5), dtype)
    add_y = to_dev(np.random.default_rng(6).normal(size=(1,) + og.sino_shape), dtype)
    s_dev = torch.tensor([0.75], device="cuda")
    got = to_np(forward_fused(g, x, op_scale=2.0, op_scale_dev=s_dev, add=add_y, add_scale=-0.5))
    ref = 1.5 * O.forward(og, to_np(x)) - 0.5 * to_np(add_y)
    assert _gate(got, ref, dtype), rel_l2(got, ref)
    y = to_dev(np.random.default_rng(7).normal(size=(1,) + og.sino_shape), dtype)
    add_x = to_dev(np.random.default_rng(8).normal(size=(1, g.n, g.n)), dtype)
    got_b = to_np(backward_fused(g, y, op_scale=-1.0, add=add_x, add_scale=1.0))
    ref_b = to_np(add_x) - O.adjoint(og, to_np(y))
    assert _gate(got_b, ref_b, dtype), rel_l2(got_b, ref_b)


def test_batch_one_agrees_with_the_batched_and_workspace_free_paths():
    g, og = make("parallel_n256_sub")
    x2 = to_dev(phantoms(g.n, 2, seed=9))
    single = to_np(forward_raw(g, x2[:1]))
    batched = to_np(forward_raw(g, x2))[:1]
    no_ws = to_np(forward_raw(g, x2[:1], workspace=None))
    ref = O.forward(og, to_np(x2[:1]))
    for got in (single, batched, no_ws):
        assert rel_l2(got, ref) <= TOL_F32
    y2 = to_dev(np.random.default_rng(10).normal(size=(2,) + og.sino_shape))
    single_b = to_np(backward_raw(g, y2[:1]))
    batched_b = to_np(backward_raw(g, y2))[:1]
    ref_b = O.adjoint(og, to_np(y2[:1]))
    for got in (single_b, batched_b):
        assert rel_l2(got, ref_b) <= TOL_F32


def test_batch_one_replays_in_a_cuda_graph():
    g, og = make("fan_ragged")
    x = to_dev(phantoms(g.n, 1, seed=13))
    y = torch.empty((1,) + g.sino_shape, device="cuda")
    xb = torch.empty_like(x)
    ws = torch.empty(L.radon_forward_workspace_size(g.handle, L.RADON_F32, 1), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        forward_raw(g, x, out=y, workspace=ws)
        backward_raw(g, y, out=xb)
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=stream):
            forward_raw(g, x, out=y, workspace=ws)
            backward_raw(g, y, out=xb)
    x.mul_(-2.0)
    graph.replay()
    torch.cuda.synchronize()
    got_y, got_x = y.clone(), xb.clone()
    forward_raw(g, x, out=y, workspace=ws)
    backward_raw(g, y, out=xb)
    torch.cuda.synchronize()
    assert torch.equal(got_y, y) and torch.equal(got_x, xb)
    assert rel_l2(to_np(got_y), O.forward(og, to_np(x))) <= TOL_F32


@pytest.mark.parametrize("dtype,texel", [(L.RADON_F32, 16), (L.RADON_F16, 8), (L.RADON_BF16, 8)])
def test_batch_one_workspace_holds_the_quad_texels(dtype, texel):
    for case in ("parallel_n64_full", "one_pixel", "fan_ragged"):
        g, _ = make(case)
        need = 2 * (g.n + 3) * (g.n + 4 + g.n % 2) * texel
        assert L.radon_forward_workspace_size(g.handle, dtype, 1) >= need
