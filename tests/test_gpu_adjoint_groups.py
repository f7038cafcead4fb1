"""Packed adjoint image groups: a CTA applies each weight it computes to 8, 16 or 32 images of the batch
(32 for larger batches where that is cheaper and the staging fits shared memory).  Every group size
sums each image's terms in the same order, so all give the same bits; the default matches the FP64
oracle on a ragged batch (a partly filled last group)."""

from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as O
from gpu_cases import TOL_F32, make, rel_l2, to_dev, to_np, within_16
from paper_2009_14788_gb300 import _lib as L, backward_raw, launch_config

pytestmark = pytest.mark.gpu


def _ws(og, batch):
    """A workspace for groups of 8, 16 or 32 images (the automatic one is sized for the default group):
    FP32 rows of a group of bg images take bg + 4 words, at most 1.5 words per image slot."""
    return torch.empty((batch + 31) // 32 * 32 * og.sino_shape[0] * og.sino_shape[1] * 6, dtype=torch.uint8,
                       device="cuda")


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16], ids=["f32", "f16", "bf16"])
@pytest.mark.parametrize("batch", [32, 33])
def test_group_sizes_give_the_same_bits_and_match_the_oracle(batch, dtype):
    g, og = make("parallel_n64_full")
    y = to_dev(np.random.default_rng(batch).normal(size=(batch,) + og.sino_shape), dtype)
    ws = _ws(og, batch)
    outs = {bg: backward_raw(g, y, launch_config(images_per_cta=bg), workspace=ws) for bg in (8, 16, 32)}
    default = backward_raw(g, y)
    for bg in (16, 32):
        assert torch.equal(outs[bg], outs[8]), bg
    assert torch.equal(default, outs[8])
    ref = O.adjoint(og, to_np(y))
    got = to_np(default)
    if dtype == torch.float32:
        assert rel_l2(got, ref) <= TOL_F32
    else:
        assert within_16(got, ref, dtype)


def test_fan_group_of_32_matches_16():
    g, og = make("fan_ragged")
    y = to_dev(np.random.default_rng(5).normal(size=(40,) + og.sino_shape), torch.float16)
    ws = _ws(og, 40)
    a = backward_raw(g, y, launch_config(images_per_cta=32), workspace=ws)
    b = backward_raw(g, y, launch_config(images_per_cta=16), workspace=ws)
    assert torch.equal(a, b)


@pytest.mark.parametrize("batch", [17, 32, 33, 64])
def test_workspace_holds_the_chosen_groups(batch):
    """The workspace size follows the group the default picks: whole groups of 8, 16 or 32 images,
    every view and detector, rows of the storage type (16-bit rows hold the group's values as they
    are; FP32 rows carry four padding words)."""
    g, og = make("fan_ragged")
    vd = og.sino_shape[0] * og.sino_shape[1]
    need16 = int(L.radon_backward_workspace_size(g.handle, L.RADON_F16, batch))
    assert need16 % (vd * 2) == 0
    slots = need16 // (vd * 2)
    assert slots >= batch and any(slots % bg == 0 and slots - batch < bg for bg in (8, 16, 32))
    need32 = int(L.radon_backward_workspace_size(g.handle, L.RADON_F32, batch))
    assert any(need32 == -(-batch // bg) * vd * (bg + 4) * 4 for bg in (8, 16, 32))
