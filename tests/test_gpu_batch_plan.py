"""Uneven batches in one persistent launch (Section 4.1, mixed sizes and geometries) against the
FP64 oracle: every item of a plan, in both directions and with both forward kernels (the staged one
and the L1 gather), in FP32 (rel-L2 1e-5) and 16-bit storage (2e-3); tile shapes that do not change
a single bit; CUDA-graph replay; and the full 64-image mixed workload with one complete item per image
size checked against the oracle."""

from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle as O
from gpu_cases import TOL_16, TOL_F32, rel_l2, to_dev, to_np, within_16
from paper_2009_14788_gb300 import BatchPlan, Geometry, _lib as L
from synth import WORKLOADS, ellipse_phantom, uneven_items, uniform_angles, workload_geometry_args, workload_images

pytestmark = pytest.mark.gpu

# a small mixed set: sizes that span several tiles and ragged tails, both geometries, odd counts
MIXED = [
    dict(kind="parallel", n=64, angles=uniform_angles(37, math.pi), det_count=91, det_spacing=1.0),
    dict(kind="parallel", n=33, angles=uniform_angles(90, math.pi) + 0.01, det_count=47, det_spacing=1.0),
    dict(kind="fan", n=48, angles=uniform_angles(29, 2 * math.pi) + 0.2, det_count=77, source_distance=130.0,
         det_distance=70.0),
    dict(kind="parallel", n=17, angles=uniform_angles(11, math.pi) + 0.3, det_count=25, det_spacing=0.9, step=0.8),
    dict(kind="parallel", n=1, angles=uniform_angles(5, math.pi), det_count=3),
    dict(kind="fan", n=80, angles=uniform_angles(45, 2 * math.pi), det_count=130, det_spacing=1.3,
         source_distance=200.0, det_distance=150.0),
]
BATCH = [1, 2, 1, 3, 1, 1]


def _geoms(args):
    a = dict(args)
    kind = a.pop("kind")
    return Geometry(kind, **a), O.Geometry.from_args(args)


def _mixed(dtype, direction, seed=0):
    rng = np.random.default_rng(seed)
    gs, ins, refs, outs = [], [], [], []
    for k, (args, b) in enumerate(zip(MIXED, BATCH)):
        g, og = _geoms(args)
        if direction == "forward":
            x = np.stack([ellipse_phantom(g.n, 5, 100 * seed + 10 * k + i) for i in range(b)])
            xin = to_dev(x, dtype)
            refs.append(O.forward(og, to_np(xin)))
            outs.append(torch.empty((b,) + og.sino_shape, dtype=dtype, device="cuda"))
        else:
            y = rng.normal(size=(b,) + og.sino_shape)
            xin = to_dev(y, dtype)
            refs.append(O.adjoint(og, to_np(xin)))
            outs.append(torch.empty((b, g.n, g.n), dtype=dtype, device="cuda"))
        gs.append(g)
        ins.append(xin)
    return gs, ins, outs, refs


# plan kinds: the staged forward, the L1-gather forward, the adjoint
KINDS = [("forward", "staged"), ("forward", "gather"), ("adjoint", "auto")]
# the shapes a tuned plan may pick: views per item (or chunk) and rows per staged slab (0: the gather)
PICKS = {("forward", "staged"): ((2, 4, 8), (16, 32)), ("forward", "gather"): ((1, 2, 4, 8), (0,)),
         ("forward", "auto"): ((1, 2, 4, 8), (0, 16, 32)), ("adjoint", "auto"): ((4, 8, 16, 32), (0,))}


@pytest.mark.parametrize("direction,kernel", KINDS + [("forward", "auto")],
                         ids=["fwd_staged", "fwd_gather", "adjoint", "fwd_auto"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16], ids=["f32", "f16", "bf16"])
def test_plan_matches_oracle(direction, kernel, dtype):
    gs, ins, outs, refs = _mixed(dtype, direction)
    plan = BatchPlan(list(zip(gs, ins, outs)), direction, forward_kernel=kernel)
    plan.launch()
    torch.cuda.synchronize()
    for k, (o, r) in enumerate(zip(outs, refs)):
        if dtype == torch.float32:
            assert rel_l2(to_np(o), r) <= TOL_F32, k
        else:
            assert within_16(to_np(o), r, dtype), (k, rel_l2(to_np(o), r))
    info = plan.info
    assert info["units"] == sum(BATCH) and info["work_items"] > 0 and info["direction"] == direction
    assert info["ctas"] % torch.cuda.get_device_properties(0).multi_processor_count == 0
    views, rows = PICKS[(direction, kernel)]
    assert all(plan.item_config(k) in views for k in range(len(gs)))
    assert all(plan.item_rows(k) in rows for k in range(len(gs)))
    assert L.radon_get_device_error(torch.cuda.current_stream().cuda_stream) == L.RADON_OK


@pytest.mark.parametrize("direction,kernel", KINDS, ids=["fwd_staged", "fwd_gather", "adjoint"])
def test_tile_shapes_do_not_change_a_bit(direction, kernel):
    """Every views-per-item (or chunk) candidate computes each output in the same order: the same bits.
    The forward's lanes per ray change only the order of a ray's partial sums, and the staged
    forward's rows per slab only where each ray's positions are re-based (FP32 rounding)."""
    gs, ins, outs, refs = _mixed(torch.float32, direction, seed=3)
    if direction == "forward":
        views = (1, 2, 4, 8)
        shapes = [(lanes, rows) for lanes in (1, 4) for rows in ((8, 16, 32) if kernel == "staged" else (0,))]
    else:
        views, shapes = (4, 8, 16, 32), [(0, 0)]
    firsts = []
    for lanes, rows in shapes:
        results = []
        for v in views:
            if direction == "forward":
                kw = dict(forward_views=v, forward_lanes=lanes, forward_rows=rows, forward_kernel=kernel)
            else:
                kw = dict(adjoint_views=v)
            plan = BatchPlan(list(zip(gs, ins, outs)), direction, autotune=False, **kw)
            assert all(plan.item_config(k) == v for k in range(len(gs)))
            assert all(plan.item_shape(k) == (v, lanes if direction == "forward" else 1) for k in range(len(gs)))
            assert all(plan.item_rows(k) == rows for k in range(len(gs)))
            plan.launch()
            torch.cuda.synchronize()
            results.append([o.clone() for o in outs])
            assert L.radon_get_device_error(torch.cuda.current_stream().cuda_stream) == L.RADON_OK
        for other in results[1:]:
            for a, b in zip(results[0], other):
                assert torch.equal(a, b)
        firsts.append(results[0])
    for res in firsts[1:]:
        for a, b, r in zip(firsts[0], res, refs):
            assert rel_l2(to_np(a), to_np(b)) <= 1e-6
            assert rel_l2(to_np(b), r) <= TOL_F32


@pytest.mark.parametrize("kernel", ["staged", "gather"])
def test_staged_and_gather_forwards_agree(kernel):
    """The two forward kernels sample the same points with the same bilinear arithmetic; they differ
    only where positions are re-based (FP32 rounding)."""
    gs, ins, outs, refs = _mixed(torch.float32, "forward", seed=9)
    BatchPlan(list(zip(gs, ins, outs)), "forward", forward_kernel=kernel).launch()
    torch.cuda.synchronize()
    mine = [o.clone() for o in outs]
    other = "gather" if kernel == "staged" else "staged"
    BatchPlan(list(zip(gs, ins, outs)), "forward", forward_kernel=other).launch()
    torch.cuda.synchronize()
    for a, b, r in zip(mine, outs, refs):
        assert rel_l2(to_np(a), to_np(b)) <= 1e-6
        assert rel_l2(to_np(a), r) <= TOL_F32


def test_tuning_cache_records_and_reuses_the_picks(tmp_path, monkeypatch):
    """With RADON_TUNE_CACHE set, a plan appends one pick per (direction, storage, size, kind, kernel)
    group and a later plan of the same groups takes its shapes from the file."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("RADON_TUNE_CACHE", str(cache))
    gs, ins, outs, refs = _mixed(torch.float32, "forward", seed=7)
    first = BatchPlan(list(zip(gs, ins, outs)), "forward", forward_kernel="staged")
    lines = cache.read_text().split("\n")
    groups = {(g.n, g.kind) for g in gs}
    assert len([l for l in lines if l.strip()]) == len(groups)
    picks = [(first.item_shape(k), first.item_rows(k)) for k in range(len(gs))]
    # rewrite the cache with other (valid) picks: a new plan must follow the file, not retime
    alt = {}
    with open(cache, "w") as f:
        for l in lines:
            if l.strip():
                key, v, ln, r = l.split()
                assert key.endswith("_staged") and int(r) in (16, 32)
                nv, nl, nr = (2 if int(v) != 2 else 4), int(ln), (32 if int(r) == 16 else 16)
                alt[key] = ((nv, nl), nr)
                f.write("%s %d %d %d\n" % (key, nv, nl, nr))
    second = BatchPlan(list(zip(gs, ins, outs)), "forward", forward_kernel="staged")
    got = [(second.item_shape(k), second.item_rows(k)) for k in range(len(gs))]
    assert sorted(set(got)) == sorted(set(alt.values())) and got != picks
    second.launch()
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert rel_l2(to_np(o), r) <= TOL_F32


@pytest.mark.parametrize("direction,kernel", KINDS, ids=["fwd_staged", "fwd_gather", "adjoint"])
def test_plan_replays_in_a_cuda_graph(direction, kernel):
    gs, ins, outs, _ = _mixed(torch.float16, direction, seed=5)
    plan = BatchPlan(list(zip(gs, ins, outs)), direction, forward_kernel=kernel)
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        plan.launch()          # warm up on the capture stream
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=stream):
            plan.launch()
    for rep in range(2):
        for t in ins:
            t.mul_(1.5 if rep == 0 else -0.25)   # new inputs, same buffers
        graph.replay()
        torch.cuda.synchronize()
        got = [o.clone() for o in outs]
        plan.launch()
        torch.cuda.synchronize()
        for a, b in zip(got, outs):
            assert torch.equal(a, b)


def test_empty_and_zero_batch_items():
    g, _ = _geoms(MIXED[0])
    x = torch.zeros((0, g.n, g.n), dtype=torch.float32, device="cuda")
    y = torch.zeros((0,) + g.sino_shape, dtype=torch.float32, device="cuda")
    plan = BatchPlan([(g, x, y)], "forward")
    assert plan.info["units"] == 0 and plan.info["work_items"] == 0
    plan.launch()
    empty = BatchPlan([], "adjoint")
    empty.launch()
    torch.cuda.synchronize()


def test_mismatched_items_are_refused():
    g, _ = _geoms(MIXED[0])
    x = torch.zeros((1, g.n, g.n), dtype=torch.float32, device="cuda")
    y16 = torch.zeros((1,) + g.sino_shape, dtype=torch.float16, device="cuda")
    with pytest.raises(ValueError):
        BatchPlan([(g, x, y16)], "forward")
    with pytest.raises(ValueError):
        BatchPlan([(g, x, torch.zeros((2,) + g.sino_shape, device="cuda"))], "forward")


def _full_uneven():
    w = WORKLOADS["uneven_b64_n128-1024"]
    items = uneven_items(w)
    geoms = []
    for k in range(len(items)):
        a = workload_geometry_args(w, k)
        kind = a.pop("kind")
        geoms.append(Geometry(kind, **a))
    return w, items, geoms


def test_staged_shapes_leave_no_bounds_flag_on_the_uneven_images():
    """One image of each size of the uneven workload (sparse to dense views, view groups across the
    class boundaries and across 90 degrees) through every staged shape: the kernel's own bounds checks
    never fire, and each result agrees with the L1 gather's."""
    w, items, geoms = _full_uneven()
    imgs = workload_images(w)
    stream = torch.cuda.current_stream().cuda_stream
    assert L.radon_get_device_error(stream) == L.RADON_OK
    for n in w.extra["sizes"]:
        k = [i for i in range(len(items)) if items[i]["n"] == n][1]
        g = geoms[k]
        x = to_dev(imgs[k][None], torch.float16)
        ref = torch.empty((1,) + g.sino_shape, dtype=torch.float16, device="cuda")
        BatchPlan([(g, x, ref)], "forward", forward_kernel="gather").launch()
        y = torch.empty_like(ref)
        for views in (2, 4, 8):
            for lanes in (1, 4):
                for rows in (8, 16, 32):
                    BatchPlan([(g, x, y)], "forward", autotune=False, forward_views=views, forward_lanes=lanes,
                              forward_rows=rows, forward_kernel="staged").launch()
                    assert L.radon_get_device_error(stream) == L.RADON_OK, (n, views, lanes, rows)
                    assert rel_l2(to_np(y), to_np(ref)) <= 1e-3, (n, views, lanes, rows)


def test_full_uneven_workload_one_item_per_size_against_oracle():
    """All 64 images (16 each of 128^2 .. 1024^2, own view counts) in one forward plan and one adjoint
    plan, fp16; for each image size the item with the fewest views is checked whole against the oracle,
    and every output is finite and non-trivial."""
    w, items, geoms = _full_uneven()
    imgs = workload_images(w)
    xs = [to_dev(x[None], torch.float16) for x in imgs]
    sinos = [torch.empty((1,) + g.sino_shape, dtype=torch.float16, device="cuda") for g in geoms]
    fwd = BatchPlan(list(zip(geoms, xs, sinos)), "forward")
    fwd.launch()
    # the adjoint's inputs: seeded sinograms drawn on the host (never the GPU's own forward output)
    rng = np.random.default_rng(6000)
    ys = [to_dev(rng.uniform(0.0, 1.0, (1,) + g.sino_shape), torch.float16) for g in geoms]
    backs = [torch.empty((1, g.n, g.n), dtype=torch.float16, device="cuda") for g in geoms]
    adj = BatchPlan(list(zip(geoms, ys, backs)), "adjoint")
    adj.launch()
    torch.cuda.synchronize()
    for k in range(len(items)):
        assert torch.isfinite(sinos[k]).all() and torch.isfinite(backs[k]).all()
    for n in w.extra["sizes"]:
        ks = [k for k in range(len(items)) if items[k]["n"] == n]
        k = min(ks, key=lambda i: items[i]["n_views"])
        og = O.Geometry.from_args(workload_geometry_args(w, k))
        ref_y = O.forward(og, to_np(xs[k]))
        assert rel_l2(to_np(sinos[k]), ref_y) <= TOL_16, (n, k)
        ref_x = O.adjoint(og, to_np(ys[k]))
        assert rel_l2(to_np(backs[k]), ref_x) <= TOL_16, (n, k)
