"""Every call documented as capturable runs inside a CUDA graph: captured once, replayed with new
inputs written into the same buffers, it gives the same bits as eager launches (no allocation, no
synchronisation, no host-side state read at replay time)."""

from __future__ import annotations

import math

import numpy as np
import pytest
import torch

from gpu_cases import make, phantoms, to_dev
from paper_2009_14788_gb300 import (Geometry, backward_fused, backward_raw, backward_workspace_bytes, cgne,
                                    filter_sinogram, forward_fused, forward_raw, forward_workspace_bytes,
                                    power_iteration)
from synth import uniform_angles

pytestmark = pytest.mark.gpu


def _capture(fn):
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        fn()                              # warm up on the capture stream
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            fn()
    torch.cuda.synchronize()
    return g


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16], ids=["f32", "f16", "bf16"])
def test_projections_replay_bit_exact(dtype):
    g, _ = make("fan_n512_block")
    x = to_dev(phantoms(g.n, 9, seed=1), dtype)
    y = forward_raw(g, x)
    oy, ox = torch.empty_like(y), torch.empty_like(x)
    fws = torch.empty(forward_workspace_bytes(g, dtype, 9), dtype=torch.uint8, device="cuda")
    bws = torch.empty(backward_workspace_bytes(g, dtype, 9), dtype=torch.uint8, device="cuda")
    alpha = torch.tensor([0.25], device="cuda")

    def step():
        forward_raw(g, x, out=oy, workspace=fws)
        backward_raw(g, y, out=ox, workspace=bws)
        backward_fused(g, oy, op_scale=-1.0, op_scale_dev=alpha, add=x, add_scale=1.0, out=ox, workspace=bws)

    graph = _capture(step)
    for rep in range(2):
        x.copy_(to_dev(phantoms(g.n, 9, seed=10 + rep), dtype))
        y.mul_(0.5)
        graph.replay()
        torch.cuda.synchronize()
        got_y, got_x = oy.clone(), ox.clone()
        step()
        torch.cuda.synchronize()
        assert torch.equal(got_y, oy) and torch.equal(got_x, ox)


def test_filter_power_iteration_and_cgne_replay_bit_exact():
    ang = uniform_angles(48, math.pi)
    g = Geometry("parallel", 64, ang, det_count=91)
    x = to_dev(phantoms(64, 2, seed=4))
    y = forward_raw(g, x)
    q = torch.empty_like(y)
    v0 = to_dev(np.random.default_rng(0).standard_normal((64, 64)))
    x0 = torch.zeros_like(x)
    res = {}

    def step():
        filter_sinogram(g, y, "hann", out=q)
        res["lam"], res["alpha"] = power_iteration(g, v0, 5)
        res["x"] = cgne(g, x0, y, 4)
        res["r"] = forward_fused(g, res["x"], add=y, add_scale=-1.0)

    graph = _capture(step)       # the outputs allocated during capture live in the graph's pool
    y.mul_(1.5)
    graph.replay()
    torch.cuda.synchronize()
    got = [q.clone(), res["lam"].clone(), res["x"].clone(), res["r"].clone()]
    step()
    torch.cuda.synchronize()
    for a, b in zip(got, [q, res["lam"], res["x"], res["r"]]):
        assert torch.equal(a, b)
