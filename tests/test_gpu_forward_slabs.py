"""The packed forward streams only the slabs that hold its rays' samples.

Each CTA of the packed forward reduces, over its rays, the first and last slab of the compute frame in
which a ray has a sample, and its producer copies only those slabs (a CTA whose rays all miss the
image copies none).  A slab outside that range gives no ray a sample, so the projection must be the
same bits as the repacking tiled forward, which streams every slab of the frame with the same
per-ray arithmetic, at the same views per CTA and rows per slab -- and meet the oracle's gates.
"""

import numpy as np
import pytest
import torch

import oracle as O
from gpu_cases import TOL_F32, make, rel_l2, to_dev, to_np, within_16
from paper_2009_14788_gb300 import _lib as L, forward_images_per_cta, forward_raw, launch_config

pytestmark = pytest.mark.gpu

DTYPES = [torch.float32, torch.float16, torch.bfloat16]
CASES = ["fan_n512_block", "fan_n512_sub", "parallel_n256_sub", "parallel_n64_full", "parallel_axes",
         "fan_close", "parallel_fine", "one_ray"]
SHAPES = [(8, 16), (4, 8), (2, 32), (1, 16)]   # views per CTA, rows per slab


def _clean():
    assert L.radon_get_device_error(torch.cuda.current_stream().cuda_stream) == L.RADON_OK


def _forward(g, x, cfg, workspace="auto"):
    """The forward of x and the number of kernels it launched, or (None, 0) where no tiled kernel
    takes the shape (a band wider than a TMA box, or shared memory)."""
    n0 = L.radon_kernel_launch_count()
    try:
        y = forward_raw(g, x, cfg, workspace=workspace)
    except L.RadonError as e:
        if e.status != L.RADON_ERR_UNSUPPORTED:
            raise
        return None, 0
    torch.cuda.synchronize()
    return y, L.radon_kernel_launch_count() - n0


def _both(g, x, cfg):
    """(packed, repacking tiled) forward of x at one shape; None for a kernel that does not take it.
    The packed path is the one that launches two kernels (the packing pass, then the projection)."""
    packed, launches = _forward(g, x, cfg)
    tiled, _ = _forward(g, x, cfg, workspace=None)
    return (packed if launches == 2 else None), tiled


@pytest.mark.parametrize("dtype", DTYPES, ids=["f32", "f16", "bf16"])
@pytest.mark.parametrize("case", CASES)
def test_packed_forward_equals_the_full_slab_stream(case, dtype):
    g, og = make(case)
    rng = np.random.default_rng(41)
    x = to_dev(rng.uniform(0.0, 1.0, (3, g.n, g.n)), dtype)
    ref = O.forward(og, to_np(x))
    compared = 0
    for views, rows in SHAPES:
        packed, tiled = _both(g, x, launch_config("tiled", views_per_cta=views, rows_per_slab=rows))
        if packed is None:
            continue
        if dtype == torch.float32:
            assert rel_l2(to_np(packed), ref) <= TOL_F32, (views, rows)
        else:
            assert within_16(to_np(packed), ref, dtype), (views, rows, rel_l2(to_np(packed), ref))
        if tiled is not None:
            assert torch.equal(packed, tiled), (views, rows)
            compared += 1
    _clean()
    if compared == 0:
        pytest.skip("the packed and the repacking forward share none of these shapes here")


def test_fp16_weight_mode_equals_the_full_slab_stream():
    g, _ = make("fan_n512_block")
    x = to_dev(np.random.default_rng(42).uniform(0.0, 1.0, (5, g.n, g.n)), torch.float16)
    packed, tiled = _both(g, x, launch_config("tiled", views_per_cta=4, rows_per_slab=16, weights=2))
    assert packed is not None and tiled is not None
    assert torch.equal(packed, tiled)
    _clean()


def test_full_size_headline_geometry_equals_the_full_slab_stream():
    """The 16 x 512^2 fan batch (720 views x 1024 detectors; about a quarter of its CTAs see no
    pixel, and about half of the slabs in all hold no sample): the library's default packed launch (8
    views per CTA, two image groups per CTA, 14 rows per slab) equals the repacking kernel that
    streams every slab at the same shape, bit for bit."""
    from paper_2009_14788_gb300 import Geometry
    from synth import WORKLOADS, workload_geometry_args
    a = workload_geometry_args(WORKLOADS["fan_b16_n512_v720_d1024"])
    kind = a.pop("kind")
    g = Geometry(kind, **a)
    x = to_dev(np.random.default_rng(43).uniform(0.0, 1.0, (16, g.n, g.n)), torch.float16)
    default = forward_raw(g, x)
    packed, tiled = _both(g, x, launch_config("tiled", views_per_cta=8, rows_per_slab=14))
    assert packed is not None and tiled is not None
    assert torch.equal(default, packed)
    assert torch.equal(packed, tiled)
    _clean()
    g.close()


@pytest.mark.parametrize("dtype", DTYPES, ids=["f32", "f16", "bf16"])
@pytest.mark.parametrize("batch", [3, 16, 20])
def test_two_image_groups_per_cta_give_the_same_bits(dtype, batch):
    """images_per_cta = two texel groups: each sample's position, floor and weights serve both groups'
    planes, every image keeps its own sum in the same order, so the projection equals the one-group
    launch bit for bit -- including a last CTA whose second group lies past the batch (read as zeros,
    never stored)."""
    g, og = make("fan_n512_block")
    bg = 4 if dtype == torch.float32 else 8
    x = to_dev(np.random.default_rng(44).uniform(0.0, 1.0, (batch, g.n, g.n)), dtype)
    compared = 0
    for views, rows in [(8, 8), (4, 16), (8, 14)]:
        one, l1 = _forward(g, x, launch_config("tiled", views_per_cta=views, rows_per_slab=rows, images_per_cta=bg))
        two, l2 = _forward(g, x, launch_config("tiled", views_per_cta=views, rows_per_slab=rows,
                                               images_per_cta=2 * bg))
        if one is None or two is None or l1 != 2 or l2 != 2:
            continue
        assert torch.equal(one, two), (views, rows)
        compared += 1
    _clean()
    assert compared > 0
    if dtype == torch.float16:
        one_w, _ = _forward(g, x, launch_config("tiled", views_per_cta=8, rows_per_slab=8, images_per_cta=8,
                                                weights=2))
        two_w, _ = _forward(g, x, launch_config("tiled", views_per_cta=8, rows_per_slab=8, images_per_cta=16,
                                                weights=2))
        assert one_w is not None and torch.equal(one_w, two_w)
    ref = O.forward(og, to_np(x[:3]))
    if dtype == torch.float32:
        assert rel_l2(to_np(two[:3]), ref) <= TOL_F32
    else:
        assert within_16(to_np(two[:3]), ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES, ids=["f32", "f16", "bf16"])
@pytest.mark.parametrize("batch", [3, 16])
def test_sparse_views_take_two_lanes_per_ray(dtype, batch):
    """Every 30th view of the fan (15 degrees apart, 1024 detectors over a 512^2 image): no CTA of 256
    detector rays has a band that fits one TMA box, so two lanes share each ray (128 rays per CTA:
    narrower bands), each summing every other sample of every slab, and the packed path still serves
    the call (a packing pass and the projection) within the oracle's gates."""
    g, og = make("fan_n512_sub")
    assert forward_images_per_cta(g, dtype, batch) == (4 if dtype == torch.float32 else 8)
    x = to_dev(np.random.default_rng(45).uniform(0.0, 1.0, (batch, g.n, g.n)), dtype)
    y, launches = _forward(g, x, launch_config())
    assert launches == 2
    ref = O.forward(og, to_np(x))
    if dtype == torch.float32:
        assert rel_l2(to_np(y), ref) <= TOL_F32
    else:
        assert within_16(to_np(y), ref, dtype)
    _clean()
