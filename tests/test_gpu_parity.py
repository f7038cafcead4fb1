"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Sizes span several tiles and ragged tails; degenerate geometries (one ray, a 1x1 image,
axis-aligned views, steep fans, very fine / coarse detectors) are included.  Gates: FP32
rel-L2 <= 1e-5 and element-wise error <= 2e-5 of the largest value; dot test <= 1e-5;
16-bit storage rel-L2 <= 2e-3 against the oracle on the storage-rounded input.
"""

import numpy as np
import pytest
import torch

import oracle as O
from gpu_cases import (CASES, TOL_16, TOL_DOT, TOL_F32, make, max_rel, phantoms, rel_l2, to_dev, to_np)
from paper_2009_14788_gb300 import Radon, RadonFanbeam, _lib as L, backward_raw, forward_raw, launch_config
from paper_2009_14788_gb300.build import build

pytestmark = pytest.mark.gpu

ALGOS = ["plain", "auto"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _rand_images(n, batch, seed):
    return np.random.default_rng(seed).uniform(0.0, 1.0, (batch, n, n))


def _rand_sino(shape, batch, seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, (batch,) + tuple(shape))


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("case", sorted(CASES))
def test_forward_matches_oracle(case, algo):
    g, og = make(case)
    x = _rand_images(g.n, 3, 11)
    ref = O.forward(og, x)
    got = to_np(forward_raw(g, to_dev(x), launch_config(algo)))
    assert got.shape == ref.shape
    assert rel_l2(got, ref) <= TOL_F32
    assert max_rel(got, ref) <= 2 * TOL_F32


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("case", sorted(CASES))
def test_backward_matches_oracle(case, algo):
    g, og = make(case)
    y = _rand_sino(g.sino_shape, 3, 12)
    ref = O.adjoint(og, y)
    got = to_np(backward_raw(g, to_dev(y), launch_config(algo)))
    assert got.shape == ref.shape
    assert rel_l2(got, ref) <= TOL_F32
    assert max_rel(got, ref) <= 2 * TOL_F32


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("case", ["parallel_n64_full", "fan_n512_sub", "parallel_ragged", "fan_steep"])
def test_dot_product_on_gpu(case, algo):
    """<A x, y> = <x, A^T y> with non-negative x, y (the gate), and with zero-mean x, y relative to
    |A x| |y| (zero-mean data cancel in the inner product, so it is not a relative scale)."""
    g, _ = make(case)
    rng = np.random.default_rng(3)
    cfg = launch_config(algo)
    x = to_dev(rng.uniform(0.0, 1.0, (2, g.n, g.n)))
    y = to_dev(rng.uniform(0.0, 1.0, (2,) + g.sino_shape))
    a = float((forward_raw(g, x, cfg).double() * y.double()).sum())
    b = float((x.double() * backward_raw(g, y, cfg).double()).sum())
    assert abs(a - b) / max(abs(a), abs(b)) <= TOL_DOT
    x = to_dev(rng.standard_normal((2, g.n, g.n)))
    y = to_dev(rng.standard_normal((2,) + g.sino_shape))
    ax = forward_raw(g, x, cfg).double()
    a = float((ax * y.double()).sum())
    b = float((x.double() * backward_raw(g, y, cfg).double()).sum())
    assert abs(a - b) / (float(ax.norm()) * float(y.double().norm())) <= 1e-6


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("case", ["parallel_n64_full", "fan_n512_sub", "parallel_ragged", "fan_ragged"])
def test_16bit_storage(case, algo, dtype):
    """16-bit in / out, FP32 arithmetic.  Kernel-only error (oracle on the rounded input) is gated;
    the end-to-end error (oracle on the FP64 input) is reported."""
    g, og = make(case)
    x = phantoms(g.n, 2)
    xs = to_dev(x, dtype)
    cfg = launch_config(algo)
    got = to_np(forward_raw(g, xs, cfg))
    kernel_only = rel_l2(got, O.forward(og, to_np(xs)))
    end_to_end = rel_l2(got, O.forward(og, x))
    assert kernel_only <= TOL_16, (kernel_only, end_to_end)
    assert end_to_end <= 2 * TOL_16, (kernel_only, end_to_end)
    y = O.forward(og, x)
    ys = to_dev(y / max(1.0, np.abs(y).max()), dtype)
    got_b = to_np(backward_raw(g, ys, cfg))
    assert rel_l2(got_b, O.adjoint(og, to_np(ys))) <= TOL_16


def test_batch_zero_and_leading_dims():
    g, og = make("parallel_ragged")
    empty = torch.zeros((0, g.n, g.n), device="cuda")
    assert forward_raw(g, empty).shape == (0,) + g.sino_shape
    x = _rand_images(g.n, 6, 5).reshape(2, 3, g.n, g.n)
    got = to_np(forward_raw(g, to_dev(x)))
    assert got.shape == (2, 3) + g.sino_shape
    assert rel_l2(got.reshape(6, *g.sino_shape), O.forward(og, x.reshape(6, g.n, g.n))) <= TOL_F32
    y = _rand_sino(g.sino_shape, 4, 6).reshape(2, 2, *g.sino_shape)
    gotb = to_np(backward_raw(g, to_dev(y)))
    assert gotb.shape == (2, 2, g.n, g.n)


def test_outputs_overwrite_not_accumulate():
    g, og = make("fan_ragged")
    x = to_dev(_rand_images(g.n, 2, 1))
    y = torch.full((2,) + g.sino_shape, 123.0, device="cuda")
    forward_raw(g, x, out=y)
    assert rel_l2(to_np(y), O.forward(og, to_np(x))) <= TOL_F32


def test_device_error_word_clear_after_normal_launches():
    g, _ = make("parallel_n64_full")
    forward_raw(g, to_dev(_rand_images(g.n, 1, 2)))
    assert L.radon_get_device_error(torch.cuda.current_stream().cuda_stream) == L.RADON_OK


# ---------------------------------------------------------------- autograd (Section 2)

def test_autograd_least_squares_gradient_matches_oracle():
    """d/dx ||A x - y||^2 = 2 A^T (A x - y), through backward() on the 256^2 geometry (views subset)."""
    g, og = make("parallel_n256_sub")
    rng = np.random.default_rng(21)
    xt = phantoms(g.n, 2, seed=30)
    y = O.forward(og, xt) + 0.01 * rng.standard_normal((2,) + g.sino_shape)
    x0 = phantoms(g.n, 2, seed=40)
    op = Radon(g.n, g.angles, det_count=g.det_count)
    x = to_dev(x0).requires_grad_(True)
    loss = ((op.forward(x) - to_dev(y)) ** 2).sum()
    loss.backward()
    ref = 2.0 * O.adjoint(og, O.forward(og, x0) - y)
    assert rel_l2(to_np(x.grad), ref) <= TOL_F32 * 10   # residual cancellation in FP32


def test_autograd_backprojection_gradient_is_forward():
    g, og = make("fan_ragged")
    op = RadonFanbeam(g.n, g.angles, source_distance=g.source_distance, det_distance=g.det_distance,
                      det_count=g.det_count, det_spacing=g.det_spacing)
    y = to_dev(_rand_sino(g.sino_shape, 2, 8)).requires_grad_(True)
    w = _rand_images(g.n, 2, 9)
    (op.backprojection(y) * to_dev(w)).sum().backward()
    assert rel_l2(to_np(y.grad), O.forward(og, w)) <= TOL_F32


def test_autograd_finite_difference_smoke():
    """FP32 directional finite difference of ||A x||^2 (loose gate: FP32 differencing)."""
    g, _ = make("parallel_n64_full")
    op = Radon(g.n, g.angles, det_count=g.det_count)
    x = to_dev(_rand_images(g.n, 1, 4)).requires_grad_(True)
    (op(x) ** 2).sum().backward()
    dirn = to_dev(np.random.default_rng(5).standard_normal((1, g.n, g.n)))
    eps = 1e-2
    with torch.no_grad():
        fp = float((op(x + eps * dirn).double() ** 2).sum())
        fm = float((op(x - eps * dirn).double() ** 2).sum())
    fd = (fp - fm) / (2 * eps)
    an = float((x.grad.double() * dirn.double()).sum())
    assert abs(fd - an) / abs(an) <= 1e-2


# ---------------------------------------------------------------- full sizes, sampled

def _full(name):
    from synth import WORKLOADS, workload_geometry_args
    from paper_2009_14788_gb300 import Geometry
    args = workload_geometry_args(WORKLOADS[name])
    a = dict(args)
    kind = a.pop("kind")
    return args, Geometry(kind, **a)


def _sampled_views(args, views):
    a = dict(args)
    a["angles"] = np.asarray(args["angles"])[views]
    return O.Geometry.from_args(a)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
@pytest.mark.parametrize("name,batch_check", [("parallel_b32_n256_v256_d363", [0, 31]),
                                              ("fan_b16_n512_v720_d1024", [0, 15])])
def test_full_size_sampled(name, batch_check, dtype):
    """Full workload batch through the tuned path; the oracle recomputes a few views of a few images
    (rays depend only on their own view angle), and the adjoint of a sinogram supported on those
    views is compared at every pixel."""
    from synth import WORKLOADS, workload_images
    args, g = _full(name)
    w = WORKLOADS[name]
    x = workload_images(w)
    xs = to_dev(x, dtype)
    y = forward_raw(g, xs)
    views = [0, 1, g.n_angles // 3, g.n_angles // 2 + 7, g.n_angles - 1]
    og = _sampled_views(args, views)
    xr = to_np(xs[batch_check])
    got = to_np(y[batch_check][:, views])
    tol = TOL_F32 if dtype == torch.float32 else TOL_16
    assert rel_l2(got, O.forward(og, xr)) <= tol
    ysp = torch.zeros_like(y)
    ysp[:, views] = y[:, views]
    xb = backward_raw(g, ysp)
    ref_b = O.adjoint(og, to_np(ysp[batch_check][:, views]))
    assert rel_l2(to_np(xb[batch_check]), ref_b) <= tol


@pytest.mark.parametrize("name", ["parallel_b32_n256_v256_d363", "fan_b16_n512_v720_d1024"])
def test_full_size_dot_product(name):
    _, g = _full(name)
    rng = np.random.default_rng(9)
    b = 4
    x = to_dev(rng.uniform(0.0, 1.0, (b, g.n, g.n)))
    y = to_dev(rng.uniform(0.0, 1.0, (b,) + g.sino_shape))
    a1 = float((forward_raw(g, x).double() * y.double()).sum())
    a2 = float((x.double() * backward_raw(g, y).double()).sum())
    assert abs(a1 - a2) / max(abs(a1), abs(a2)) <= TOL_DOT


def test_sample_count_is_the_throughput_unit():
    args, g = _full("parallel_b32_n256_v256_d363")
    assert g.sample_count == O.sample_count(O.Geometry.from_args(args))
    assert g.sample_count > 256 * 256 * 250


# ---------------------------------------------------------------- tiled kernels: explicit configurations

TILED_CASES = ["parallel_n64_full", "parallel_n256_sub", "fan_n512_block", "parallel_axes", "fan_close",
               "parallel_fine", "parallel_coarse", "fan_ragged", "parallel_ragged", "one_ray", "one_pixel"]


@pytest.mark.parametrize("ws", ["packed", "staged"])
@pytest.mark.parametrize("images", [4, 8, 16])
@pytest.mark.parametrize("batch", [1, 5, 17])
@pytest.mark.parametrize("case", ["fan_n512_sub", "parallel_ragged", "fan_close"])
def test_backward_tiled_image_groups(case, batch, images, ws):
    """Every images-per-CTA setting with full, ragged and single-image batches, with a workspace
    (sinogram packed once; 8 or 16 images per CTA) and without (per-CTA staging; 4, 8 or 16)."""
    if ws == "packed" and images == 4:
        pytest.skip("the packed adjoint groups 8 or 16 images")
    g, og = make(case)
    y = _rand_sino(g.sino_shape, batch, 40 + batch)
    got = to_np(backward_raw(g, to_dev(y), launch_config("tiled", images_per_cta=images),
                             workspace="auto" if ws == "packed" else None))
    ref = O.adjoint(og, y)
    assert rel_l2(got, ref) <= TOL_F32
    assert max_rel(got, ref) <= 2 * TOL_F32


@pytest.mark.parametrize("ws", ["packed", "staged"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16])
@pytest.mark.parametrize("case", TILED_CASES)
def test_backward_tiled_bounds_word_stays_clear(case, dtype, ws):
    """The tiled adjoint's own window check never fires, and results match the oracle."""
    g, og = make(case)
    y = _rand_sino(g.sino_shape, 3, 50)
    ys = to_dev(y, dtype)
    got = to_np(backward_raw(g, ys, launch_config("tiled"), workspace="auto" if ws == "packed" else None))
    assert L.radon_get_device_error(torch.cuda.current_stream().cuda_stream) == L.RADON_OK
    tol = TOL_F32 if dtype == torch.float32 else TOL_16
    assert rel_l2(got, O.adjoint(og, to_np(ys))) <= tol


def test_tiled_refuses_extreme_magnification_and_auto_falls_back():
    """Source 50 px from the centre of a 64^2 image: a 16^2 tile projects onto hundreds of detector
    bins, more than one TMA box; TILED reports it, AUTO serves it with the plain kernel."""
    g, og = make("fan_steep")
    y = _rand_sino(g.sino_shape, 2, 60)
    with pytest.raises(L.RadonError, match="TMA box"):
        backward_raw(g, to_dev(y), launch_config("tiled"))
    with pytest.raises(L.RadonError, match="TMA box"):
        backward_raw(g, to_dev(y), launch_config("tiled"), workspace=None)
    assert rel_l2(to_np(backward_raw(g, to_dev(y))), O.adjoint(og, y)) <= TOL_F32


def test_backward_tiled_unsupported_is_reported():
    """A misaligned sinogram cannot be staged by TMA: TILED says so, AUTO serves it with the plain kernel."""
    g, og = make("parallel_n64_full")
    y = _rand_sino(g.sino_shape, 1, 3)
    buf = torch.zeros(int(np.prod(g.sino_shape)) + 1, device="cuda")
    view = buf[1:].view(1, *g.sino_shape)
    view.copy_(to_dev(y))
    with pytest.raises(L.RadonError):
        backward_raw(g, view, launch_config("tiled"), workspace=None)
    got = to_np(backward_raw(g, view, launch_config("auto"), workspace=None))
    assert rel_l2(got, O.adjoint(og, y)) <= TOL_F32


FWD_TILED_CASES = [c for c in TILED_CASES if CASES[c]["n"] % 8 == 0]


WS = ["packed", "repack"]   # forward with a workspace (batch packed once) / without (per-CTA repack)


def _ws(kind):
    return "auto" if kind == "packed" else None


@pytest.mark.parametrize("ws", WS)
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16])
@pytest.mark.parametrize("case", FWD_TILED_CASES)
def test_forward_tiled_matches_oracle(case, dtype, ws):
    """TMA-staged slab forward, every storage type, both input paths; ragged image group."""
    g, og = make(case)
    x = _rand_images(g.n, 3, 70)
    xs = to_dev(x, dtype)
    got = to_np(forward_raw(g, xs, launch_config("tiled"), workspace=_ws(ws)))
    assert L.radon_get_device_error(torch.cuda.current_stream().cuda_stream) == L.RADON_OK
    ref = O.forward(og, to_np(xs))
    if dtype == torch.float32:
        assert rel_l2(got, ref) <= TOL_F32
        assert max_rel(got, ref) <= 2 * TOL_F32
    else:
        assert rel_l2(got, ref) <= TOL_16


@pytest.mark.parametrize("ws", WS)
@pytest.mark.parametrize("rows", [2, 8, 16])
@pytest.mark.parametrize("views", [1, 2, 4, 8])
@pytest.mark.parametrize("case", ["fan_n512_block", "parallel_n256_sub", "fan_close"])
def test_forward_tiled_configs(case, views, rows, ws):
    g, og = make(case)
    x = _rand_images(g.n, 9, 80)
    cfg = launch_config("tiled", views_per_cta=views, rows_per_slab=rows)
    try:
        got = to_np(forward_raw(g, to_dev(x), cfg, workspace=_ws(ws)))
    except L.RadonError as exc:
        # a configuration whose working band exceeds one TMA box is refused, never run
        assert exc.status == L.RADON_ERR_UNSUPPORTED and "TMA box" in str(exc)
        return
    assert L.radon_get_device_error(torch.cuda.current_stream().cuda_stream) == L.RADON_OK
    ref = O.forward(og, x)
    assert rel_l2(got, ref) <= TOL_F32
    assert max_rel(got, ref) <= 2 * TOL_F32


@pytest.mark.parametrize("ws", WS)
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16], ids=["f32", "f16", "bf16"])
@pytest.mark.parametrize("case", ["fan_n512_block", "parallel_n64_full"])
def test_forward_paired_view_phases_give_the_same_bits(case, dtype, ws):
    """Closely spaced views ((n / 2) |theta_{v+1} - theta_v| <= 5 pixels): CTAs of 2 to 8 views give
    each 8-lane load phase two views x four detectors, a CTA of one view cannot.  Every ray sums the
    same samples in the same order either way, so all shapes give the same bits, and match the oracle."""
    g, og = make(case)
    xs = to_dev(_rand_images(g.n, 9, 81), dtype)
    outs = []
    for v in (1, 2, 4, 8):
        try:
            outs.append(forward_raw(g, xs, launch_config("tiled", views_per_cta=v, rows_per_slab=16),
                                    workspace=_ws(ws)))
        except L.RadonError as exc:   # a working band wider than one TMA box is refused, never run
            assert exc.status == L.RADON_ERR_UNSUPPORTED and "TMA box" in str(exc) and v == 1
    assert len(outs) >= 3
    assert L.radon_get_device_error(torch.cuda.current_stream().cuda_stream) == L.RADON_OK
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    ref = O.forward(og, to_np(xs))
    got = to_np(outs[-1])
    if dtype == torch.float32:
        assert rel_l2(got, ref) <= TOL_F32
    else:
        assert rel_l2(got, ref) <= TOL_16


def test_forward_sparse_wide_views_take_two_lanes_per_ray():
    """Every 30th view of the 512^2 fan set (15 degrees apart): no CTA of one thread per ray keeps the
    working band inside one TMA box.  An explicit views per CTA (one thread per ray) is refused; left
    to the library, two threads share each ray (half the detectors per CTA) and the packed kernel
    serves the request, TILED and AUTO alike."""
    g, og = make("fan_n512_sub")
    x = _rand_images(g.n, 2, 91)
    with pytest.raises(L.RadonError, match="TMA box"):
        forward_raw(g, to_dev(x), launch_config("tiled", views_per_cta=8))
    for cfg in (launch_config("tiled"), None):
        assert rel_l2(to_np(forward_raw(g, to_dev(x), cfg)), O.forward(og, x)) <= TOL_F32


@pytest.mark.parametrize("case", ["parallel_ragged", "fan_ragged", "one_pixel"])
def test_forward_tiled_refuses_unaligned_rows_auto_serves(case):
    """Image rows that are not a multiple of 16 bytes cannot be described to TMA: TILED says so,
    AUTO serves the request with the plain kernel."""
    g, og = make(case)
    x = _rand_images(g.n, 2, 90)
    with pytest.raises(L.RadonError, match="16 bytes"):
        forward_raw(g, to_dev(x), launch_config("tiled"), workspace=None)
    assert rel_l2(to_np(forward_raw(g, to_dev(x))), O.forward(og, x)) <= TOL_F32


def test_forward_workspace_too_small_uses_paths_without_one():
    g, og = make("fan_n512_block")
    x = _rand_images(g.n, 5, 93)
    from paper_2009_14788_gb300 import forward_workspace_bytes
    need = forward_workspace_bytes(g, torch.float32, 5)
    assert need == 2 * 2 * g.n * g.n * 16          # 2 groups of 4 images, rows + transposed copy
    small = torch.empty(need - 16, dtype=torch.uint8, device="cuda")
    got = to_np(forward_raw(g, to_dev(x), workspace=small))
    assert rel_l2(got, O.forward(og, x)) <= TOL_F32


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("case", ["parallel_ragged", "fan_ragged", "one_pixel", "parallel_coarse"])
def test_forward_packed_any_image_size(case, dtype):
    """The packed path addresses 16-byte texels, so image sides that are not a multiple of 16
    bytes (97, 75, 1, 60 in 16-bit) still take the tiled kernel."""
    g, og = make(case)
    x = _rand_images(g.n, 3, 94)
    xs = to_dev(x, dtype)
    got = to_np(forward_raw(g, xs, launch_config("tiled"), workspace="auto"))
    assert L.radon_get_device_error(torch.cuda.current_stream().cuda_stream) == L.RADON_OK
    ref = O.forward(og, to_np(xs))
    assert rel_l2(got, ref) <= (TOL_F32 if dtype == torch.float32 else TOL_16)


@pytest.mark.parametrize("ws", WS)
@pytest.mark.parametrize("case", FWD_TILED_CASES)
def test_fp16_weight_modes(case, ws):
    """FP16 storage: FP32 bilinear weights (the default) and FP16 weights in mixed-precision FMAs
    (weights=2, opt-in) both meet the 16-bit gate, and per ray they differ by no more than the
    weights' rounding (relative <= 2^-12 each, so <= 2^-12 of the ray sum for non-negative images)
    plus one FP16 output rounding of each result (2^-11 each).  weights=1 names the default."""
    g, og = make(case)
    x = phantoms(g.n, 3)
    xs = to_dev(x, torch.float16)
    ref = O.forward(og, to_np(xs))
    fast = to_np(forward_raw(g, xs, launch_config("tiled", weights=2), workspace=_ws(ws)))
    exact = to_np(forward_raw(g, xs, launch_config("tiled"), workspace=_ws(ws)))
    named = to_np(forward_raw(g, xs, launch_config("tiled", weights=1), workspace=_ws(ws)))
    assert np.array_equal(exact, named)
    assert rel_l2(fast, ref) <= TOL_16 and rel_l2(exact, ref) <= TOL_16
    bound = (2.0 ** -12 + 2 * 2.0 ** -11) * np.abs(ref) + 1e-6 * np.abs(ref).max()
    assert np.all(np.abs(fast - exact) <= bound)
