"""Failure detection on the GPU without a GPU fault: a bounded wait that nothing completes.

RADON_TEST_STALL_TMA=1 makes the tiled adjoint issue no copies, so its first bounded mbarrier
wait expires; the kernel records RADON_ERR_TIMEOUT in the device error word and returns.  The
host reads the status, and the context stays usable for the next call.
"""

import numpy as np
import pytest
import torch

from gpu_cases import TOL_F32, make, rel_l2, to_dev, to_np
from paper_2009_14788_gb300 import _lib as L, backward_raw, launch_config
from paper_2009_14788_gb300.build import build

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def test_bounded_wait_expiry_is_reported_and_context_survives(monkeypatch):
    g, og = make("parallel_n64_full")
    y = np.random.default_rng(1).uniform(-1, 1, (2,) + g.sino_shape)
    stream = torch.cuda.current_stream().cuda_stream
    assert L.radon_get_device_error(stream) == L.RADON_OK
    monkeypatch.setenv("RADON_TEST_STALL_TMA", "1")
    backward_raw(g, to_dev(y), launch_config("tiled"), workspace=None)
    assert L.radon_get_device_error(stream) == L.RADON_ERR_TIMEOUT
    assert "bounded wait" in L.radon_last_error_message()
    monkeypatch.delenv("RADON_TEST_STALL_TMA")
    # the word was cleared by the read, and the next launch works normally
    got = to_np(backward_raw(g, to_dev(y), launch_config("tiled")))
    assert L.radon_get_device_error(stream) == L.RADON_OK
    assert rel_l2(got, O.adjoint(og, y)) <= TOL_F32
