"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle comparisons.

This package holds input generation only (phantoms, angle sets, noise, workload
recipes). It contains none of the Radon arithmetic: both the CUDA path and the
FP64 oracle consume what it produces, and neither imports the other.
"""

from .phantoms import (  # noqa: F401
    EllipseSpec,
    random_ellipses,
    rasterize_ellipses,
    ellipse_phantom,
    gaussian_blob,
    uniform_angles,
)
from .workloads import (  # noqa: F401
    WORKLOADS, Workload, power_start, uneven_items, workload_geometry_args, workload_images, workload_noise)
