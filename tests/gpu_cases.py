"""Shared geometry cases and comparison helpers for the GPU parity tests."""

from __future__ import annotations

import math

import numpy as np
import torch

import oracle as O
from paper_2009_14788_gb300 import Geometry
from synth import WORKLOADS, ellipse_phantom, uniform_angles, workload_geometry_args

# FP32 gates (rel-L2 against the FP64 oracle) and the 16-bit gate, per the stated targets.
TOL_F32 = 1e-5
TOL_DOT = 1e-5
TOL_16 = 2e-3


def _sub(args, views):
    a = dict(args)
    a["angles"] = np.asarray(a["angles"])[views]
    return a


CASES = {
    # the 64^2 workload at full size
    "parallel_n64_full": workload_geometry_args(WORKLOADS["parallel_b1_n64_v64_d91"]),
    # the 256^2 workload, every 8th view
    "parallel_n256_sub": _sub(workload_geometry_args(WORKLOADS["parallel_b32_n256_v256_d363"]), slice(0, None, 8)),
    # the 512^2 fan workload, every 30th view
    "fan_n512_sub": _sub(workload_geometry_args(WORKLOADS["fan_b16_n512_v720_d1024"]), slice(0, None, 30)),
    # the 512^2 fan workload, 24 consecutive views (a contiguous block of the dense view set)
    "fan_n512_block": _sub(workload_geometry_args(WORKLOADS["fan_b16_n512_v720_d1024"]), slice(100, 124)),
    # ragged sizes, non-unit spacing and step
    "parallel_ragged": dict(kind="parallel", n=97, angles=uniform_angles(13, math.pi) + 0.03, det_count=150,
                            det_spacing=0.83, step=0.7),
    "fan_ragged": dict(kind="fan", n=75, angles=uniform_angles(17, 2 * math.pi) + 0.3, det_count=101,
                       source_distance=120.0, det_distance=60.0),
    # axis-aligned and diagonal views: samples land exactly on pixel lattices
    "parallel_axes": dict(kind="parallel", n=48, angles=np.array([0.0, math.pi / 4, math.pi / 2, math.pi,
                                                                  1.25 * math.pi, 1.5 * math.pi]),
                          det_count=70, det_spacing=1.0),
    # degenerate: one detector, one view; and a 1x1 image
    "one_ray": dict(kind="parallel", n=40, angles=np.array([0.37]), det_count=1),
    "one_pixel": dict(kind="parallel", n=1, angles=uniform_angles(5, math.pi), det_count=3),
    # steep fan: wide fan angle, detector far away, rays up to ~40 degrees off the central ray
    "fan_steep": dict(kind="fan", n=64, angles=uniform_angles(11, 2 * math.pi), det_count=200, det_spacing=2.0,
                      source_distance=50.0, det_distance=300.0),
    # a close source (magnification up to ~4 across the image) that the tiled kernels still take
    "fan_close": dict(kind="fan", n=64, angles=uniform_angles(13, 2 * math.pi) + 0.05, det_count=160,
                      det_spacing=1.2, source_distance=70.0, det_distance=90.0),
    # detector spacing much finer and much coarser than a pixel
    "parallel_fine": dict(kind="parallel", n=40, angles=uniform_angles(9, math.pi) + 0.1, det_count=200,
                          det_spacing=0.3, step=0.5),
    "parallel_coarse": dict(kind="parallel", n=60, angles=uniform_angles(9, math.pi) + 0.1, det_count=25,
                            det_spacing=3.1, step=1.9),
    # a pixel's candidate window just under three rays wide at the diagonal views (2 sqrt(2) / 0.955
    # = 2.96): the widest windows that the single-image adjoint's three-candidate stepping takes
    "parallel_three_rays": dict(kind="parallel", n=50, angles=np.array([0.1, math.pi / 4, 0.9, 3 * math.pi / 4,
                                                                         2.0, 2.6]),
                                det_count=80, det_spacing=0.955),
}


def make(case: str):
    args = CASES[case]
    a = dict(args)
    kind = a.pop("kind")
    return Geometry(kind, **a), O.Geometry.from_args(args)


def phantoms(n: int, batch: int, seed: int = 7) -> np.ndarray:
    return np.stack([ellipse_phantom(n, 6, seed + b) for b in range(batch)])


def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def ulp16(ref, dtype) -> np.ndarray:
    """One unit in the last place of ``dtype`` (float16 / bfloat16) at each |ref|."""
    a = np.maximum(np.abs(np.asarray(ref, dtype=np.float64)), 1e-30)
    e = np.floor(np.log2(a))
    bits = 10 if dtype == torch.float16 else 7
    if dtype == torch.float16:
        e = np.maximum(e, -14.0)   # subnormal spacing below 2^-14
    return np.exp2(e - bits)


def within_16(got, ref, dtype) -> bool:
    """The 16-bit storage gate.  rel-L2 <= 2e-3 bounds the RMS of many independent roundings; an
    output of fewer than 64 elements is gated element-wise at one storage ulp instead (a single
    correctly rounded bfloat16 value may be 2^-8 = 3.9e-3 off in relative terms)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if got.size >= 64:
        return rel_l2(got, ref) <= TOL_16
    return bool(np.all(np.abs(got - ref) <= ulp16(ref, dtype) * (1 + 1e-9)))


def max_rel(got, ref) -> float:
    """Element-wise: worst |got - ref| relative to the largest |ref|."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def to_dev(a: np.ndarray, dtype=torch.float32) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().to(torch.float64).cpu().numpy()
