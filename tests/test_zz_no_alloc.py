"""radon_forward_static_scratch: the forward projection for callers that cannot allocate.

Real-time loops that forbid allocation after start-up, code that must not let an allocation
synchronise the device, and plain C hosts without a device allocator cannot provide the scratch
workspace that the packed forward path needs.  This entry point keeps that scratch in a fixed 32 MiB
array inside the library.  Its results must meet the FP64 oracle's gate and equal those of the
workspace-taking entry point (radon_forward_ws) on consecutive calls -- the array is shared and
overwritten by every call -- and requests that do not fit must be refused.

This file is collected last, so a run that stops at the first failure has run every other test.
"""

import numpy as np
import pytest
import torch

import oracle as O
from gpu_cases import TOL_F32, TOL_16, make, rel_l2, to_dev, to_np
from paper_2009_14788_gb300 import _lib as L, forward_workspace_bytes
from paper_2009_14788_gb300.build import build

pytestmark = pytest.mark.gpu

_DT = {torch.float32: L.RADON_F32, torch.float16: L.RADON_F16, torch.bfloat16: L.RADON_BF16}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _with_workspace(g, x):
    """The existing entry point: radon_forward_ws with a caller workspace."""
    batch = x.shape[0]
    y = torch.empty((batch,) + g.sino_shape, dtype=x.dtype, device="cuda")
    ws = torch.empty(forward_workspace_bytes(g, x.dtype, batch), dtype=torch.uint8, device="cuda")
    st = L.radon_forward_ws(g.handle, x.data_ptr(), y.data_ptr(), _DT[x.dtype], batch, None, ws.data_ptr(),
                            ws.numel(), torch.cuda.current_stream().cuda_stream)
    L.check(st, "radon_forward_ws")
    return y


def _static(g, x):
    batch = x.shape[0]
    y = torch.full((batch,) + g.sino_shape, float("nan"), dtype=x.dtype, device="cuda")
    st = L.radon_forward_static_scratch(g.handle, x.data_ptr(), y.data_ptr(), _DT[x.dtype], batch,
                                        torch.cuda.current_stream().cuda_stream)
    L.check(st, "radon_forward_static_scratch")
    return y


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16])
@pytest.mark.parametrize("case", ["fan_n512_block", "parallel_ragged"])
def test_static_scratch_matches_oracle_and_workspace_entry_point_twice(case, dtype):
    """Two calls in a row with different inputs and batch sizes (the shared array is reused): each
    meets the FP64 oracle's gate on the storage-rounded input, and equals the workspace-taking entry
    point bit for bit (same pack and packed kernel; batches of two or more)."""
    g, og = make(case)
    rng = np.random.default_rng(7)
    tol = TOL_F32 if dtype == torch.float32 else TOL_16
    for call, batch in enumerate((5, 3)):
        x = to_dev(rng.uniform(0.0, 1.0, (batch, g.n, g.n)), dtype)
        got = to_np(_static(g, x))
        assert np.all(np.isfinite(got)), "call %d left outputs unwritten" % call
        assert rel_l2(got, O.forward(og, to_np(x))) <= tol, "call %d" % call
        assert np.array_equal(got, to_np(_with_workspace(g, x))), "call %d" % call
    assert L.radon_get_device_error(torch.cuda.current_stream().cuda_stream) == L.RADON_OK


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_static_scratch_single_image_matches_oracle(dtype):
    """A batch of one runs the same packed path (one group with one image): checked against the
    oracle, twice with different images."""
    g, og = make("fan_n512_block")
    rng = np.random.default_rng(11)
    for call in range(2):
        x = to_dev(rng.uniform(0.0, 1.0, (1, g.n, g.n)), dtype)
        got = to_np(_static(g, x))
        assert rel_l2(got, O.forward(og, to_np(x))) <= (TOL_F32 if dtype == torch.float32 else TOL_16), call


def test_static_scratch_refuses_batches_beyond_its_size():
    g, _ = make("fan_n512_block")
    x = torch.zeros((1, g.n, g.n), device="cuda")
    y = torch.zeros((1,) + g.sino_shape, device="cuda")
    big = 64   # 64 float32 images of 512^2 need 2 x 16 groups x 512^2 x 16 B = 128 MiB of scratch
    assert forward_workspace_bytes(g, torch.float32, big) > (32 << 20)
    st = L.radon_forward_static_scratch(g.handle, x.data_ptr(), y.data_ptr(), L.RADON_F32, big,
                                        torch.cuda.current_stream().cuda_stream)
    assert st == L.RADON_ERR_INVALID_ARG
    assert "static scratch" in L.radon_last_error_message()
