"""The exact adjoint with a precomputed weight table (radon_geometry_build_adjoint_table).

The table holds, per 16 x 16 tile, view and pixel pair, the weights that the packed adjoint computes on
the fly, computed by the same arithmetic; the adjoint that reads them adds the same nonzero products in
the same order.  So its results must equal the table-free adjoint bit for bit (and meet the FP64
oracle's gates), for every storage type and for the 8- and 16-image groups that it serves (batches
of more than 16 images run 16-image groups while a table exists).  Geometries whose pixel pairs weigh on rays spanning more than
five detectors in a view keep computing their weights for those views (the table marks them); only
geometries the packed adjoint cannot serve are refused.
"""

import numpy as np
import pytest
import torch

import oracle as O
from gpu_cases import TOL_16, TOL_F32, make, rel_l2, to_dev, to_np, within_16
from paper_2009_14788_gb300 import _lib as L, backward_raw

pytestmark = pytest.mark.gpu

DTYPES = [torch.float32, torch.float16, torch.bfloat16]
CASES = ["fan_n512_block", "fan_n512_sub", "parallel_n256_sub", "parallel_ragged", "fan_ragged", "parallel_axes",
         "parallel_three_rays", "parallel_fine", "parallel_coarse", "fan_close", "one_ray", "one_pixel"]


def _clean():
    assert L.radon_get_device_error(torch.cuda.current_stream().cuda_stream) == L.RADON_OK


@pytest.mark.parametrize("dtype", DTYPES, ids=["f32", "f16", "bf16"])
@pytest.mark.parametrize("case", CASES)
def test_table_adjoint_equals_the_gather_bit_for_bit(case, dtype):
    g, og = make(case)
    rng = np.random.default_rng(31)
    ys = {b: to_dev(rng.normal(size=(b,) + g.sino_shape), dtype) for b in (3, 16)}
    want = {b: backward_raw(g, y) for b, y in ys.items()}   # packed adjoint, weights on the fly
    g.build_adjoint_table()
    try:
        for b, y in ys.items():
            got = backward_raw(g, y)
            torch.cuda.synchronize()
            assert torch.equal(got, want[b]), (case, b)
            ref = O.adjoint(og, to_np(y))
            if dtype == torch.float32:
                assert rel_l2(to_np(got), ref) <= TOL_F32, (case, b)
            else:
                assert within_16(to_np(got), ref, dtype), (case, b, rel_l2(to_np(got), ref))
        _clean()
    finally:
        g.free_adjoint_table()
    # freed: the weights are computed again, the same bits
    assert torch.equal(backward_raw(g, ys[3]), want[3])


def test_table_serves_larger_batches_and_leaves_single_images_alone():
    """With a table, batches of more than 16 images run 16-image groups that read it instead of
    32-image groups that compute their weights (one pixel per thread); batch-1 calls keep their own
    kernel.  The same bits either way."""
    g, og = make("fan_n512_sub")
    rng = np.random.default_rng(5)
    y40 = to_dev(rng.normal(size=(40,) + g.sino_shape), torch.float16)
    y1 = to_dev(rng.normal(size=(1,) + g.sino_shape), torch.float32)
    a40, a1 = backward_raw(g, y40), backward_raw(g, y1)
    g.build_adjoint_table()
    try:
        assert torch.equal(backward_raw(g, y40), a40)
        assert torch.equal(backward_raw(g, y1), a1)
        assert rel_l2(to_np(a1), O.adjoint(og, to_np(y1))) <= TOL_F32
        _clean()
    finally:
        g.free_adjoint_table()


def test_table_size_and_rebuild():
    g, _ = make("parallel_ragged")
    tiles = ((g.n + 15) // 16) ** 2
    assert g.adjoint_table_bytes() == tiles * g.n_angles * (128 * 44 + 4)
    y = to_dev(np.random.default_rng(2).normal(size=(5,) + g.sino_shape), torch.float32)
    want = backward_raw(g, y)
    g.build_adjoint_table()
    g.build_adjoint_table()   # replaces the first table
    try:
        assert torch.equal(backward_raw(g, y), want)
    finally:
        g.free_adjoint_table()
        g.free_adjoint_table()   # freeing twice is harmless


def test_dense_rays_overflow_to_the_computed_weights():
    """Detectors much finer than a pixel: most pairs weigh on more than four rays, the table marks
    them, and the adjoint still gives the table-free bits."""
    g, og = make("parallel_fine")
    y = to_dev(np.random.default_rng(3).normal(size=(4,) + g.sino_shape), torch.float32)
    want = backward_raw(g, y)
    assert g.adjoint_table_overflow() == 0.0
    g.build_adjoint_table()
    try:
        assert g.adjoint_table_overflow() > 0.5
        assert torch.equal(backward_raw(g, y), want)
        assert rel_l2(to_np(want), O.adjoint(og, to_np(y))) <= TOL_F32
        _clean()
    finally:
        g.free_adjoint_table()


def test_geometries_the_packed_adjoint_cannot_serve_are_refused():
    """A detector window wider than 256 rays (a steep, strongly magnifying fan): no table is kept and
    the adjoint runs as before."""
    g, og = make("fan_steep")
    with pytest.raises(L.RadonError) as ei:
        g.build_adjoint_table()
    assert ei.value.status == L.RADON_ERR_UNSUPPORTED
    assert g.adjoint_table_overflow() == 0.0
    y = to_dev(np.random.default_rng(3).normal(size=(4,) + g.sino_shape), torch.float32)
    assert rel_l2(to_np(backward_raw(g, y)), O.adjoint(og, to_np(y))) <= TOL_F32
    _clean()


def test_full_size_headline_geometry_with_table_against_oracle_on_sampled_views():
    """The 16 x 512^2 fan batch (720 views x 1024 detectors) through the table adjoint equals the
    table-free adjoint bit for bit; and a sub-geometry of every 60th view through the table meets
    the oracle's 16-bit gate."""
    from paper_2009_14788_gb300 import Geometry
    from synth import WORKLOADS, workload_geometry_args
    w = WORKLOADS["fan_b16_n512_v720_d1024"]
    a = workload_geometry_args(w)
    kind = a.pop("kind")
    g = Geometry(kind, **a)
    y = to_dev(np.random.default_rng(9).uniform(0.0, 1.0, (16,) + g.sino_shape), torch.float16)
    want = backward_raw(g, y)
    g.build_adjoint_table()
    try:
        assert g.adjoint_table_overflow() < 0.01   # spans of 2-5 rays
        assert torch.equal(backward_raw(g, y), want)
        _clean()
    finally:
        g.free_adjoint_table()
    g.close()
    sub = workload_geometry_args(w)
    sub["angles"] = np.asarray(sub["angles"])[::60]
    og = O.Geometry.from_args(sub)
    kind = sub.pop("kind")
    gs = Geometry(kind, **sub)
    ys = to_dev(np.random.default_rng(10).uniform(0.0, 1.0, (16,) + gs.sino_shape), torch.float16)
    gs.build_adjoint_table()
    try:
        got = backward_raw(gs, ys)
        assert rel_l2(to_np(got), O.adjoint(og, to_np(ys))) <= TOL_16
    finally:
        gs.free_adjoint_table()


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
def test_table_under_fused_epilogues_graphs_and_autograd(dtype):
    """The table serves every caller of the packed adjoint: a fused epilogue (device step length and
    addend, the Landweber update), a CUDA-graph replay, and the gradient of the forward projection
    through autograd -- each equal, bit for bit, to the same call without a table."""
    from paper_2009_14788_gb300 import Radon, backward_fused
    from synth import uniform_angles
    g, og = make("parallel_n256_sub")
    rng = np.random.default_rng(12)
    y = to_dev(rng.normal(size=(6,) + g.sino_shape), dtype)
    add = to_dev(rng.normal(size=(6, g.n, g.n)), dtype)
    s_dev = torch.tensor([0.37], device="cuda")

    def fused():
        return backward_fused(g, y, op_scale=-1.5, op_scale_dev=s_dev, add=add, add_scale=0.5)

    radon = Radon(64, uniform_angles(33, np.pi), det_count=91)
    x = torch.from_numpy(rng.uniform(0.0, 1.0, (6, 64, 64))).to("cuda", torch.float32)

    def grad():
        xg = x.clone().requires_grad_(True)
        (radon.forward(xg) ** 2).sum().backward()
        return xg.grad

    want_f, want_g = fused(), grad()
    stream = torch.cuda.Stream()
    g.build_adjoint_table()
    radon.build_adjoint_table()
    try:
        assert torch.equal(fused(), want_f)
        assert torch.equal(grad(), want_g)
        out = torch.empty_like(want_f)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            backward_fused(g, y, op_scale=-1.5, op_scale_dev=s_dev, add=add, add_scale=0.5, out=out)
            torch.cuda.synchronize()
            with torch.cuda.graph(graph, stream=stream):
                backward_fused(g, y, op_scale=-1.5, op_scale_dev=s_dev, add=add, add_scale=0.5, out=out)
        out.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, want_f)
        _clean()
    finally:
        g.free_adjoint_table()
        radon.geometry.free_adjoint_table()
