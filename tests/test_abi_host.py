"""libradon's C ABI on the host: it loads, exports what include/radon.h declares, rejects bad
arguments before touching a GPU, and builds geometry tables that agree with the FP64 oracle
(sample counts bit-exact, sample positions to FP32 rounding).  No GPU needed."""

import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2009_14788_gb300 import Geometry, _lib as L
from paper_2009_14788_gb300.build import build
from synth import WORKLOADS, uniform_angles, workload_geometry_args

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _header_names():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            names |= set(re.findall(r"RADON_API\s+[\w\s\*]+?\b(radon_\w+)\s*\(", open(os.path.join(inc, f)).read()))
    return names


def test_library_exports_every_declared_symbol():
    names = _header_names()
    assert len(names) >= 15
    lib = ctypes.CDLL(L.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert names == set(L.exported_names())
    assert L.radon_abi_version() == 2


def test_status_strings():
    for code, name in [(0, "RADON_OK"), (1, "RADON_ERR_INVALID_ARG"), (2, "RADON_ERR_UNSUPPORTED"),
                       (3, "RADON_ERR_OOM"), (4, "RADON_ERR_CUDA"), (5, "RADON_ERR_TIMEOUT"),
                       (6, "RADON_ERR_DEVICE_BOUNDS")]:
        assert L.status_string(code) == name
    assert L.status_string(99) == "RADON_ERR_UNKNOWN"


def _create(**kw):
    args = dict(n=16, angles=np.linspace(0, np.pi, 8, endpoint=False), n_angles=None, is_fan=0,
                source_distance=0.0, det_distance=0.0, det_count=0, det_spacing=0.0, step=0.0, host_only=1)
    args.update(kw)
    ang = np.ascontiguousarray(args["angles"], dtype=np.float64) if args["angles"] is not None else None
    desc = L.radon_geometry_desc(args["n"], ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if ang is not None
                                 else None, args["n_angles"] if args["n_angles"] is not None else ang.size,
                                 args["is_fan"], args["source_distance"], args["det_distance"], args["det_count"],
                                 args["det_spacing"], args["step"], args["host_only"])
    h = ctypes.c_void_p()
    st = L.radon_geometry_create(ctypes.byref(desc), ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("kw,code", [
    (dict(n=0), L.RADON_ERR_INVALID_ARG),
    (dict(n=9000), L.RADON_ERR_INVALID_ARG),
    (dict(angles=None, n_angles=4), L.RADON_ERR_INVALID_ARG),
    (dict(n_angles=0), L.RADON_ERR_INVALID_ARG),
    (dict(angles=np.array([0.0, np.nan])), L.RADON_ERR_INVALID_ARG),
    (dict(step=np.inf), L.RADON_ERR_INVALID_ARG),
    (dict(step=1e-5), L.RADON_ERR_INVALID_ARG),
    (dict(det_spacing=np.nan), L.RADON_ERR_INVALID_ARG),
    (dict(is_fan=1, source_distance=0.0), L.RADON_ERR_INVALID_ARG),
    (dict(is_fan=1, source_distance=10.0), L.RADON_ERR_UNSUPPORTED),   # source inside the image
    (dict(is_fan=2), L.RADON_ERR_INVALID_ARG),
])
def test_create_rejects_bad_arguments(kw, code):
    st, h = _create(**kw)
    assert st == code, L.radon_last_error_message()
    assert not h.value
    assert L.radon_last_error_message() != ""


def test_null_out_pointer():
    ang = np.zeros(2)
    st = L.radon_geometry_create_parallel(8, ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 2, 0, 0.0, 0.0,
                                          None)
    assert st == L.RADON_ERR_INVALID_ARG


def test_allocation_failure_injection(monkeypatch):
    monkeypatch.setenv("RADON_FAULT_INJECT_OOM", "1")
    st, h = _create()
    assert st == L.RADON_ERR_OOM and not h.value
    monkeypatch.delenv("RADON_FAULT_INJECT_OOM")
    st, h = _create()
    assert st == L.RADON_OK
    L.radon_geometry_destroy(h)


def test_launch_argument_checks_without_gpu():
    st, h = _create()
    assert st == L.RADON_OK
    buf = (ctypes.c_float * 4)()
    p = ctypes.addressof(buf)
    cfg = L.radon_launch_config(0, 0, 0, 0, 0, 0, 0)
    assert L.radon_forward(None, p, p + 4, 0, 1, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_forward(h, p, p + 4, 7, 1, None) == L.RADON_ERR_INVALID_ARG        # dtype
    assert L.radon_forward(h, p, p + 4, 0, -1, None) == L.RADON_ERR_INVALID_ARG       # batch
    assert L.radon_forward(h, None, p, 0, 1, None) == L.RADON_ERR_INVALID_ARG         # NULL input
    assert L.radon_backward(h, p, p, 0, 1, None) == L.RADON_ERR_INVALID_ARG           # aliasing
    cfg.threads = 48
    assert L.radon_forward_ex(h, p, p + 4, 0, 1, ctypes.byref(cfg), None) == L.RADON_ERR_INVALID_ARG
    cfg.threads = 0
    cfg.weights = 3
    assert L.radon_forward_ex(h, p, p + 4, 0, 1, ctypes.byref(cfg), None) == L.RADON_ERR_INVALID_ARG
    assert "weights" in L.radon_last_error_message()
    cfg.weights = 0
    cfg.algo = 9
    assert L.radon_backward_ex(h, p, p + 4, 0, 1, ctypes.byref(cfg), None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_forward(h, p, p + 4, 0, 1, None) == L.RADON_ERR_INVALID_ARG        # host-only geometry
    assert "host-only" in L.radon_last_error_message()
    assert L.radon_geometry_sample_count(None) == -1
    L.radon_geometry_destroy(h)
    L.radon_geometry_destroy(None)


def test_iterative_entry_points_reject_bad_arguments_without_gpu():
    st, h = _create()
    assert st == L.RADON_OK
    buf = (ctypes.c_double * 64)()
    p = ctypes.addressof(buf)
    ws_bytes = int(L.radon_dot_workspace_size())
    assert ws_bytes >= 8
    # radon_dot: dtype, count, result pointer, alignment, workspace, non-finite scale
    assert L.radon_dot(p, p, 7, 4, 1.0, p, 0, p, ws_bytes, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_dot(p, p, 0, -1, 1.0, p, 0, p, ws_bytes, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_dot(p, p, 0, 4, 1.0, None, 0, p, ws_bytes, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_dot(p + 2, p, 0, 4, 1.0, p, 0, p, ws_bytes, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_dot(None, p, 0, 4, 1.0, p, 0, p, ws_bytes, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_dot(p, p, 0, 4, 1.0, p, 0, p, ws_bytes - 8, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_dot(p, p, 0, 4, 1.0, p, 0, p + 4, ws_bytes, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_dot(p, p, 0, 4, float("inf"), p, 0, p, ws_bytes, None) == L.RADON_ERR_INVALID_ARG
    # radon_axpby: dtypes, count, NULL operands, alignment, scalars
    assert L.radon_axpby(p, 0, p, 9, 4, 1.0, None, 0.0, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_axpby(p, 0, p, 0, -2, 1.0, None, 0.0, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_axpby(None, 0, p, 0, 4, 1.0, None, 0.0, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_axpby(p + 1, 1, p, 0, 4, 1.0, None, 0.0, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_axpby(p, 0, p, 0, 4, 1.0, p + 2, 0.0, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_axpby(p, 0, p, 0, 4, float("nan"), None, 0.0, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_axpby(p, 0, p, 0, 0, 1.0, None, 0.0, None) == L.RADON_OK             # nothing to do
    # radon_power_iteration: host-only geometry, pointers, iterations, workspace
    need = int(L.radon_power_iteration_workspace_size(h))
    assert need > 0 and int(L.radon_power_iteration_workspace_size(None)) == 0
    assert L.radon_power_iteration(h, p, 20, p, None, p, need, None) == L.RADON_ERR_INVALID_ARG
    assert "host-only" in L.radon_last_error_message()
    assert L.radon_power_iteration(None, p, 20, p, None, p, need, None) == L.RADON_ERR_INVALID_ARG
    # radon_forward_fused / radon_backward_fused: misaligned addend or scalar, non-finite scales
    ep = L.radon_epilogue(1.0, None, -1.0, p + 1)
    assert L.radon_forward_fused(h, p, p + 64, 0, 1, ctypes.byref(ep), None, None, 0, None) == L.RADON_ERR_INVALID_ARG
    ep = L.radon_epilogue(1.0, p + 2, 0.0, None)
    assert L.radon_backward_fused(h, p, p + 64, 0, 1, ctypes.byref(ep), None, None, 0, None) == \
        L.RADON_ERR_INVALID_ARG
    ep = L.radon_epilogue(float("inf"), None, 0.0, None)
    assert L.radon_forward_fused(h, p, p + 64, 0, 1, ctypes.byref(ep), None, None, 0, None) == L.RADON_ERR_INVALID_ARG
    assert "finite" in L.radon_last_error_message()
    ep = L.radon_epilogue(1.0, None, 0.0, None)
    assert L.radon_forward_fused(h, p, p + 64, 0, 1, ctypes.byref(ep), None, p + 8, 0, None) == \
        L.RADON_ERR_INVALID_ARG                                                           # workspace alignment
    L.radon_geometry_destroy(h)


def test_batch_plan_rejects_bad_arguments_without_gpu():
    st, h = _create()
    assert st == L.RADON_OK
    buf = (ctypes.c_double * 16)()
    p = ctypes.addressof(buf)
    out = ctypes.c_void_p()
    items = (L.radon_item * 2)(L.radon_item(h, p, p + 64, 1), L.radon_item(h, p, p + 64, 1))
    # a host-only geometry cannot be planned
    assert L.radon_batch_plan_create(items, 2, 0, 0, None, ctypes.byref(out)) == L.RADON_ERR_INVALID_ARG
    assert "host-only" in L.radon_last_error_message() and not out.value
    assert L.radon_batch_plan_create(None, 2, 0, 0, None, ctypes.byref(out)) == L.RADON_ERR_INVALID_ARG
    assert L.radon_batch_plan_create(items, -1, 0, 0, None, ctypes.byref(out)) == L.RADON_ERR_INVALID_ARG
    assert L.radon_batch_plan_create(items, 2, 2, 0, None, ctypes.byref(out)) == L.RADON_ERR_INVALID_ARG
    assert L.radon_batch_plan_create(items, 2, 0, 5, None, ctypes.byref(out)) == L.RADON_ERR_INVALID_ARG
    assert L.radon_batch_plan_create(items, 2, 0, 0, None, None) == L.RADON_ERR_INVALID_ARG
    opts = L.radon_plan_options(1, 3, 0)
    assert L.radon_batch_plan_create(items, 2, 0, 0, ctypes.byref(opts), ctypes.byref(out)) == L.RADON_ERR_INVALID_ARG
    opts = L.radon_plan_options(1, 0, 5)
    assert L.radon_batch_plan_create(items, 2, 1, 0, ctypes.byref(opts), ctypes.byref(out)) == L.RADON_ERR_INVALID_ARG
    opts = L.radon_plan_options(1, 0, 0, 2)
    assert L.radon_batch_plan_create(items, 2, 0, 0, ctypes.byref(opts), ctypes.byref(out)) == L.RADON_ERR_INVALID_ARG
    assert "forward_lanes" in L.radon_last_error_message()
    opts = L.radon_plan_options(1, 0, 0, 0, 12)
    assert L.radon_batch_plan_create(items, 2, 0, 0, ctypes.byref(opts), ctypes.byref(out)) == L.RADON_ERR_INVALID_ARG
    assert "forward_rows" in L.radon_last_error_message()
    opts = L.radon_plan_options(1, 0, 0, 0, 0, 2)
    assert L.radon_batch_plan_create(items, 2, 0, 0, ctypes.byref(opts), ctypes.byref(out)) == L.RADON_ERR_INVALID_ARG
    assert "forward_kernel" in L.radon_last_error_message()
    bad = (L.radon_item * 1)(L.radon_item(None, p, p + 64, 1))
    assert L.radon_batch_plan_create(bad, 1, 0, 0, None, ctypes.byref(out)) == L.RADON_ERR_INVALID_ARG
    # a dead handle is refused by every plan call
    info = L.radon_plan_info()
    v = ctypes.c_int()
    assert L.radon_batch_plan_launch(None, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_batch_plan_get_info(None, ctypes.byref(info)) == L.RADON_ERR_INVALID_ARG
    assert L.radon_batch_plan_item_config(None, 0, ctypes.byref(v)) == L.RADON_ERR_INVALID_ARG
    assert L.radon_batch_plan_item_shape(None, 0, ctypes.byref(v), ctypes.byref(v)) == L.RADON_ERR_INVALID_ARG
    L.radon_batch_plan_destroy(None)
    L.radon_geometry_destroy(h)


def test_filter_rejects_bad_arguments_without_gpu():
    st, h = _create()
    assert st == L.RADON_OK
    buf = (ctypes.c_float * 64)()
    p = ctypes.addressof(buf)
    assert L.radon_filter_sinogram(h, p, p + 128, 0, 1, 9, None) == L.RADON_ERR_INVALID_ARG      # unknown filter
    assert L.radon_filter_sinogram(h, p, p + 128, 0, 1, 0, None) == L.RADON_ERR_INVALID_ARG      # host-only
    assert "host-only" in L.radon_last_error_message()
    assert L.radon_filter_sinogram(None, p, p + 128, 0, 1, 0, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_filter_sinogram(h, p, p + 128, 0, -1, 0, None) == L.RADON_ERR_INVALID_ARG
    assert sorted(L.FILTERS.values()) == list(range(5))
    L.radon_geometry_destroy(h)


def test_defaults_follow_the_paper():
    g = Geometry("parallel", 40, uniform_angles(5, math.pi), host_only=True)
    assert (g.det_count, g.det_spacing, g.step) == (40, 1.0, 1.0)
    # Section 3.1.2 worked example: S = Ddet = 512, N = D = 512 -> spacing 2.0
    f = Geometry("fan", 512, uniform_angles(4, 2 * math.pi), source_distance=512.0, host_only=True)
    assert f.det_count == 512 and f.det_distance == 512.0 and f.det_spacing == 2.0


GEOMS = {
    "parallel_even": dict(kind="parallel", n=32, angles=uniform_angles(37, math.pi) + 0.01, det_count=47),
    "parallel_axes": dict(kind="parallel", n=20, angles=np.array([0, math.pi / 4, math.pi / 2, math.pi, 1.5 * math.pi]),
                          det_count=22, det_spacing=1.0),
    "parallel_odd_spacing": dict(kind="parallel", n=33, angles=uniform_angles(29, 2 * math.pi), det_count=41,
                                 det_spacing=0.83, step=0.7),
    "fan": dict(kind="fan", n=40, angles=uniform_angles(31, 2 * math.pi) + 0.2, det_count=64, det_spacing=1.1,
                source_distance=80.0, det_distance=50.0),
    "fan_default": dict(kind="fan", n=25, angles=uniform_angles(23, 2 * math.pi), source_distance=40.0),
    "one_pixel": dict(kind="parallel", n=1, angles=uniform_angles(7, math.pi), det_count=3),
    "parallel_b1_n64": workload_geometry_args(WORKLOADS["parallel_b1_n64_v64_d91"]),
}


def _lib_geom(args):
    a = dict(args)
    kind = a.pop("kind")
    return Geometry(kind, host_only=True, **a)


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_sample_counts_match_oracle_exactly(name):
    g = _lib_geom(GEOMS[name])
    og = O.Geometry.from_args(GEOMS[name])
    _, counts = g.rays()
    np.testing.assert_array_equal(counts, O.ray_sample_counts(og))
    assert g.sample_count == O.sample_count(og)


def test_sample_counts_match_oracle_full_fan_workload_subset():
    """The 512^2 fan workload: every 24th view (FP64 enumeration must agree ray by ray)."""
    args = workload_geometry_args(WORKLOADS["fan_b16_n512_v720_d1024"])
    args["angles"] = args["angles"][::24]
    g = _lib_geom(args)
    _, counts = g.rays()
    np.testing.assert_array_equal(counts, O.ray_sample_counts(O.Geometry.from_args(args)))


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_ray_table_positions_match_oracle(name):
    """Every tabulated sample position equals an oracle sample position to FP32 rounding."""
    g = _lib_geom(GEOMS[name])
    og = O.Geometry.from_args(GEOMS[name])
    rays, counts = g.rays()
    c0 = (og.n - 1) / 2.0
    half = (og.n + 1) / 2.0
    worst = 0.0
    for v in range(og.n_angles):
        for d in range(og.det_count):
            nk = counts[v, d]
            if nk == 0:
                continue
            m, u = O.ray(og, v, d)
            ks = np.arange(-4 * og.n - 8, 4 * og.n + 9)
            t = ks * og.step
            px, py = m[0] + t * u[0], m[1] + t * u[1]
            ins = (np.abs(px) < half) & (np.abs(py) < half)
            ref = np.stack([px[ins] + c0, py[ins] + c0], axis=1)
            J0, I0, fx0, fy0, dxh, dyh, dxl, dyl = (float(z) for z in rays[v, d])
            kk = np.arange(nk)
            got = np.stack([J0 + fx0 + kk * dxh + kk * dxl, I0 + fy0 + kk * dyh + kk * dyl], axis=1)
            if len(ref) > 1 and np.dot(ref[-1] - ref[0], got[-1] - got[0]) < 0:
                ref = ref[::-1]
            assert len(ref) == nk
            assert 0.0 <= fx0 < 1.0 and 0.0 <= fy0 < 1.0
            # the high parts keep few enough bits that k * dxh is exact in FP32, including a margin of
            # 24 px / h samples past either end of the ray (the adjoint's tile reference samples)
            margin = 24 * int(np.ceil(1.0 / og.step)) + 8
            km = np.arange(-margin, nk + margin)
            for hpart in (dxh, dyh):
                assert np.all(np.float32(km * np.float32(hpart)) == km * hpart)
            assert np.all(np.isfinite(got))
            worst = max(worst, float(np.max(np.abs(got - ref))))
    assert worst < 1e-6


def test_orientation_major_axis_step_is_nonnegative():
    g = _lib_geom(GEOMS["fan"])
    rays, counts = g.rays()
    th = GEOMS["fan"]["angles"]
    vertical = np.abs(np.cos(th)) >= np.abs(np.sin(th))
    for v in range(len(th)):
        sel = counts[v] > 1
        step = (rays[v, sel, 5] + rays[v, sel, 7]) if vertical[v] else (rays[v, sel, 4] + rays[v, sel, 6])
        assert np.all(step >= 0)


def test_forward_workspace_covers_the_single_image_texels():
    """A batch-1 forward packs the image's 2 x 2 quad texels (both frames, two texels of border, an
    even row pitch of at least N + 4) into the workspace: (N + 3) rows of that pitch twice, 16 bytes
    each for FP32, 8 for 16-bit storage; larger batches keep the batch-interleaved size."""
    for n in (1, 40, 97):
        g = Geometry("parallel", n, uniform_angles(5, math.pi), host_only=True)
        for dt, texel in ((L.RADON_F32, 16), (L.RADON_F16, 8), (L.RADON_BF16, 8)):
            one = int(L.radon_forward_workspace_size(g.handle, dt, 1))
            pitch = n + 4 + (n % 2)
            assert one >= 2 * (n + 3) * pitch * texel
            two = int(L.radon_forward_workspace_size(g.handle, dt, 2))
            assert two > 0 and int(L.radon_forward_workspace_size(g.handle, dt, 0)) == 0


def test_forward_images_per_cta_on_the_host():
    """The packed forward's images per CTA, asked without a launch: 16-bit batches of more than one
    texel group (8 images) pair their groups, FP32 and single groups take one; images_per_cta picks one
    or two groups where it names one of those values (else the default); one image under AUTO and the
    PLAIN algorithm run other kernels (0)."""
    from paper_2009_14788_gb300 import forward_images_per_cta, launch_config
    import torch
    a = workload_geometry_args(WORKLOADS["fan_b16_n512_v720_d1024"])
    kind = a.pop("kind")
    g = Geometry(kind, host_only=True, **a)
    f16, bf16, f32 = torch.float16, torch.bfloat16, torch.float32
    assert forward_images_per_cta(g, f16, 16) == 16
    assert forward_images_per_cta(g, bf16, 9) == 16
    assert forward_images_per_cta(g, f16, 8) == 8
    assert forward_images_per_cta(g, f16, 2) == 8
    assert forward_images_per_cta(g, f32, 16) == 4
    assert forward_images_per_cta(g, f16, 16, launch_config(images_per_cta=8)) == 8
    assert forward_images_per_cta(g, f16, 3, launch_config(images_per_cta=16)) == 16
    assert forward_images_per_cta(g, f32, 16, launch_config(images_per_cta=8)) == 8
    assert forward_images_per_cta(g, f16, 16, launch_config(images_per_cta=32)) == 16   # an adjoint value
    assert forward_images_per_cta(g, f16, 1) == 0
    assert forward_images_per_cta(g, f16, 1, launch_config("tiled")) == 8
    assert forward_images_per_cta(g, f16, 16, launch_config("plain")) == 0
    assert forward_images_per_cta(g, f16, 0) == 0
    # sparse views widen the bands: at 8 views per CTA two groups' buffers (14 rows) exceed shared
    # memory and the default falls back to one group; asked for explicitly, two groups are refused;
    # at 2 views per CTA, or 8 rows per slab, two groups fit
    sparse = Geometry("parallel", 256, uniform_angles(8, math.pi), det_count=363, host_only=True)
    assert forward_images_per_cta(sparse, f16, 16, launch_config("tiled", views_per_cta=8)) == 8
    assert forward_images_per_cta(sparse, f16, 16, launch_config("tiled", views_per_cta=8, images_per_cta=16)) == 0
    assert forward_images_per_cta(sparse, f16, 16, launch_config("tiled", views_per_cta=2)) == 16
    assert forward_images_per_cta(sparse, f16, 16, launch_config("tiled", views_per_cta=8, rows_per_slab=8)) == 16
    # every 30th view of the fan (15 degrees apart): no one-lane shape fits a TMA box; two lanes per ray
    # (half the detectors per CTA) take one texel group at two views per CTA or one
    sub = workload_geometry_args(WORKLOADS["fan_b16_n512_v720_d1024"])
    sub["angles"] = np.asarray(sub["angles"])[::30]
    kind = sub.pop("kind")
    gs = Geometry(kind, host_only=True, **sub)
    assert forward_images_per_cta(gs, f16, 16) == 8
    assert forward_images_per_cta(gs, f32, 3) == 4
    assert forward_images_per_cta(gs, f16, 16, launch_config("tiled", views_per_cta=8)) == 0
    assert forward_images_per_cta(gs, f16, 16, launch_config(images_per_cta=16)) == 0
    n = ctypes.c_int(-1)
    assert L.radon_forward_images_per_cta(g.handle, L.RADON_F16, -1, None, ctypes.byref(n)) == L.RADON_ERR_INVALID_ARG
    assert L.radon_forward_images_per_cta(g.handle, L.RADON_F16, 4, None, None) == L.RADON_ERR_INVALID_ARG


def test_adjoint_table_size_and_refusals_on_the_host():
    """The weight table's size is a closed form of the geometry (tiles x views x (128 pairs x 44 + 4)
    bytes); a host-only geometry can be asked for it but cannot build one, and without a table the
    overflow fraction is 0."""
    for n, V in ((1, 3), (40, 7), (97, 13)):
        g = Geometry("parallel", n, uniform_angles(V, math.pi), host_only=True)
        tiles = ((n + 15) // 16) ** 2
        assert g.adjoint_table_bytes() == tiles * V * (128 * 44 + 4)
        assert g.adjoint_table_overflow() == 0.0
        st = L.radon_geometry_build_adjoint_table(g.handle)
        assert st == L.RADON_ERR_INVALID_ARG
        assert L.radon_geometry_free_adjoint_table(g.handle) == L.RADON_OK


def test_probe_arguments_are_checked_on_the_host():
    """The gather-ceiling probe refuses bad arguments before touching a GPU: a NULL result, an unknown
    storage type, a weights setting outside 0..2, FP16 weights for other storage, and texel groups other
    than 1 or 2."""
    out = ctypes.c_double(0.0)
    assert L.radon_probe_gather_ceiling_groups(L.RADON_F16, 0, 1, None) == L.RADON_ERR_INVALID_ARG
    assert L.radon_probe_gather_ceiling_groups(7, 0, 1, ctypes.byref(out)) == L.RADON_ERR_INVALID_ARG
    assert L.radon_probe_gather_ceiling_groups(L.RADON_F16, 3, 1, ctypes.byref(out)) == L.RADON_ERR_INVALID_ARG
    assert L.radon_probe_gather_ceiling_groups(L.RADON_BF16, 2, 1, ctypes.byref(out)) == L.RADON_ERR_INVALID_ARG
    for groups in (0, 3, -1):
        assert L.radon_probe_gather_ceiling_groups(L.RADON_F16, 0, groups, ctypes.byref(out)) == L.RADON_ERR_INVALID_ARG
    assert L.radon_probe_gather_ceiling_ex(L.RADON_F32, 2, ctypes.byref(out)) == L.RADON_ERR_INVALID_ARG
    assert out.value == 0.0
