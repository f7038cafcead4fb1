"""The five seeded workloads (geometry parameters + phantom recipes).

Each workload is described by plain numbers only.  ``workload_geometry_args``
returns keyword arguments that both the CUDA library's geometry constructor and
the oracle's geometry accept; ``workload_images`` returns the seeded float64
phantoms.  Seeds: phantom ``b`` of workload number ``c`` uses ``1000*c + b``;
noise uses ``2000*c``; per-image view counts of the uneven batch use ``5000``.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .phantoms import ellipse_phantom, uniform_angles


@dataclass(frozen=True)
class Workload:
    number: int            # 1..5, used only to derive seeds
    name: str
    kind: str              # "parallel" | "fan" | "landweber" | "uneven"
    n: int                 # image side (0 for the uneven batch)
    batch: int
    n_views: int
    span: float            # angles equally spaced in [0, span)
    det_count: int
    det_spacing: float
    step: float = 1.0
    source_distance: float = 0.0
    det_distance: float = 0.0
    n_ellipses: int = 10
    axes: tuple | None = None
    storage: str = "f32"
    extra: dict = field(default_factory=dict)


WORKLOADS: dict[str, Workload] = {
    w.name: w
    for w in [
        # one 64x64 image, 5 ellipses with semi-axes U[4,20]
        Workload(1, "parallel_b1_n64_v64_d91", "parallel", 64, 1, 64, math.pi, 91, 1.0,
                 n_ellipses=5, axes=(4.0, 20.0)),
        # 32 x 256^2, 256 views in [0, pi), 363 detectors; y = A x + N(0, 0.01^2)
        Workload(2, "parallel_b32_n256_v256_d363", "parallel", 256, 32, 256, math.pi, 363, 1.0,
                 extra={"noise_sigma": 0.01}),
        # 16 x 512^2 fan beam, 720 views in [0, 2 pi), S=1000, D_det=500, 1024 x 1.5
        Workload(3, "fan_b16_n512_v720_d1024", "fan", 512, 16, 720, 2 * math.pi, 1024, 1.5,
                 source_distance=1000.0, det_distance=500.0),
        # 8 x 512^2, 60 views in [0, pi), ceil(512 sqrt 2) = 725 detectors, bf16 storage
        Workload(4, "landweber_b8_n512_v60_d725", "landweber", 512, 8, 60, math.pi, 725, 1.0,
                 storage="bf16", extra={"iterations": 10, "power_iterations": 20, "noise_sigma": 0.01}),
        # 64 images, 16 each of 128/256/512/1024, own parallel geometry each, fp16 storage
        Workload(5, "uneven_b64_n128-1024", "uneven", 0, 64, 0, math.pi, 0, 1.0,
                 storage="f16", extra={"sizes": (128, 256, 512, 1024), "per_size": 16,
                                       "views_lo": 90, "views_hi": 1024}),
    ]
}


def uneven_items(w: Workload) -> list[dict]:
    """Per-image (n, n_views, det_count) of the uneven batch, seeded."""
    rng = np.random.default_rng(5000)
    items = []
    for n in w.extra["sizes"]:
        for _ in range(w.extra["per_size"]):
            v = int(rng.integers(w.extra["views_lo"], w.extra["views_hi"] + 1))
            items.append({"n": n, "n_views": v, "det_count": int(math.ceil(n * math.sqrt(2.0)))})
    return items


def workload_geometry_args(w: Workload, item: int | None = None) -> dict:
    """Constructor arguments shared by the library geometry and the oracle geometry."""
    if w.kind == "uneven":
        it = uneven_items(w)[item]
        return dict(kind="parallel", n=it["n"], angles=uniform_angles(it["n_views"], w.span),
                    det_count=it["det_count"], det_spacing=w.det_spacing, step=w.step)
    args = dict(kind="fan" if w.kind == "fan" else "parallel", n=w.n,
                angles=uniform_angles(w.n_views, w.span), det_count=w.det_count,
                det_spacing=w.det_spacing, step=w.step)
    if w.kind == "fan":
        args.update(source_distance=w.source_distance, det_distance=w.det_distance)
    return args


def workload_images(w: Workload, indices=None) -> list[np.ndarray] | np.ndarray:
    """Seeded float64 phantoms: an array [B, N, N], or a list for the uneven batch."""
    if w.kind == "uneven":
        items = uneven_items(w)
        idx = range(len(items)) if indices is None else indices
        return [ellipse_phantom(items[b]["n"], w.n_ellipses, 1000 * w.number + b, w.axes) for b in idx]
    idx = range(w.batch) if indices is None else indices
    return np.stack([ellipse_phantom(w.n, w.n_ellipses, 1000 * w.number + b, w.axes) for b in idx])


def workload_noise(w: Workload, shape) -> np.ndarray:
    sigma = w.extra.get("noise_sigma", 0.0)
    return np.random.default_rng(2000 * w.number).normal(0.0, sigma, size=shape)


def power_start(n: int, seed: int) -> np.ndarray:
    """The power method's start vector: N(0, 1) pixels from ``numpy.random.default_rng(seed)``."""
    return np.random.default_rng(seed).standard_normal((n, n))
