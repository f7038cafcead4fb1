"""GB300-native discrete Radon transform (forward projection + exact adjoint).

Fixed-step bilinear ray sampling for parallel- and fan-beam geometries, hand-written CUDA
kernels for sm_103a behind the C ABI in ``include/radon.h`` (``libradon.so``), with a thin
PyTorch binding: ``Radon``, ``RadonFanbeam``, differentiable forward / backprojection.
"""

from . import _lib  # noqa: F401
from .landweber import Landweber, LandweberFunction, landweber  # noqa: F401
from .solvers import cg, cgne  # noqa: F401
from .radon import (  # noqa: F401
    BatchPlan,
    FilterSinogramFunction,
    Geometry,
    Radon,
    RadonBackprojectionFunction,
    RadonFanbeam,
    RadonForwardFunction,
    axpby,
    backproject_interpolating,
    backward_fused,
    backward_raw,
    backward_workspace_bytes,
    dot,
    filter_sinogram,
    forward_fused,
    forward_images_per_cta,
    forward_raw,
    forward_workspace_bytes,
    launch_config,
    power_iteration,
)

__all__ = [
    "Geometry", "Radon", "RadonFanbeam", "RadonForwardFunction", "RadonBackprojectionFunction", "forward_raw",
    "backward_raw", "launch_config", "forward_workspace_bytes", "backward_workspace_bytes", "forward_fused",
    "backward_fused", "dot", "axpby", "power_iteration", "Landweber", "LandweberFunction", "landweber", "BatchPlan",
    "filter_sinogram", "FilterSinogramFunction", "cg", "cgne",
    "backproject_interpolating", "forward_images_per_cta",
]
