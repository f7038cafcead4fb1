"""ctypes binding of libradon's C ABI (include/radon.h): argument marshalling only.

Every name here is the C function of the same name.  Loading fails loudly if the shared
library has not been built: there is no fallback implementation.
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libradon.so")

RADON_OK = 0
RADON_ERR_INVALID_ARG = 1
RADON_ERR_UNSUPPORTED = 2
RADON_ERR_OOM = 3
RADON_ERR_CUDA = 4
RADON_ERR_TIMEOUT = 5
RADON_ERR_DEVICE_BOUNDS = 6

RADON_F32 = 0
RADON_F16 = 1
RADON_BF16 = 2

FILTERS = {"ram-lak": 0, "shepp-logan": 1, "cosine": 2, "hamming": 3, "hann": 4}

RADON_ALGO_AUTO = 0
RADON_ALGO_PLAIN = 1
RADON_ALGO_TILED = 2

RADON_WEIGHTS_DEFAULT = 0   # FP32 bilinear weights
RADON_WEIGHTS_F32 = 1
RADON_WEIGHTS_F16 = 2       # FP16 storage only: FP16 weights in mixed-precision FMAs (opt-in)


class RadonError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__("%s failed: %s: %s" % (where, status_string(status), message))


class radon_geometry_desc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("angles", ctypes.POINTER(ctypes.c_double)),
        ("n_angles", ctypes.c_int),
        ("is_fan", ctypes.c_int),
        ("source_distance", ctypes.c_double),
        ("det_distance", ctypes.c_double),
        ("det_count", ctypes.c_int),
        ("det_spacing", ctypes.c_double),
        ("step", ctypes.c_double),
        ("host_only", ctypes.c_int),
    ]


class radon_geometry_info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("n_angles", ctypes.c_int),
        ("det_count", ctypes.c_int),
        ("is_fan", ctypes.c_int),
        ("det_spacing", ctypes.c_double),
        ("step", ctypes.c_double),
        ("source_distance", ctypes.c_double),
        ("det_distance", ctypes.c_double),
        ("sample_count", ctypes.c_int64),
        ("device", ctypes.c_int),
    ]


class radon_launch_config(ctypes.Structure):
    _fields_ = [
        ("algo", ctypes.c_int),
        ("views_per_cta", ctypes.c_int),
        ("rows_per_slab", ctypes.c_int),
        ("images_per_cta", ctypes.c_int),
        ("tile", ctypes.c_int),
        ("threads", ctypes.c_int),
        ("weights", ctypes.c_int),
    ]


class radon_epilogue(ctypes.Structure):
    _fields_ = [
        ("op_scale", ctypes.c_float),
        ("op_scale_dev", ctypes.c_void_p),
        ("add_scale", ctypes.c_float),
        ("add", ctypes.c_void_p),
    ]


class radon_item(ctypes.Structure):
    _fields_ = [
        ("geometry", ctypes.c_void_p),
        ("in_", ctypes.c_void_p),
        ("out", ctypes.c_void_p),
        ("batch", ctypes.c_int),
    ]


class radon_plan_options(ctypes.Structure):
    _fields_ = [
        ("autotune", ctypes.c_int),
        ("forward_views", ctypes.c_int),
        ("adjoint_views", ctypes.c_int),
        ("forward_lanes", ctypes.c_int),
        ("forward_rows", ctypes.c_int),
        ("forward_kernel", ctypes.c_int),
    ]


class radon_plan_info(ctypes.Structure):
    _fields_ = [
        ("units", ctypes.c_int),
        ("work_items", ctypes.c_int),
        ("ctas", ctypes.c_int),
        ("direction", ctypes.c_int),
    ]


_c = None

# (name, restype, argtypes) of every exported function
_SIGNATURES = [
    ("radon_geometry_create_parallel", ctypes.c_int,
     [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
      ctypes.POINTER(ctypes.c_void_p)]),
    ("radon_geometry_create_fanbeam", ctypes.c_int,
     [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
      ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_void_p)]),
    ("radon_geometry_create", ctypes.c_int, [ctypes.POINTER(radon_geometry_desc), ctypes.POINTER(ctypes.c_void_p)]),
    ("radon_geometry_copy_rays", ctypes.c_int,
     [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32)]),
    ("radon_geometry_destroy", None, [ctypes.c_void_p]),
    ("radon_geometry_get_info", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(radon_geometry_info)]),
    ("radon_geometry_sample_count", ctypes.c_int64, [ctypes.c_void_p]),
    ("radon_geometry_adjoint_table_size", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    ("radon_geometry_build_adjoint_table", ctypes.c_int, [ctypes.c_void_p]),
    ("radon_geometry_free_adjoint_table", ctypes.c_int, [ctypes.c_void_p]),
    ("radon_geometry_adjoint_table_overflow", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    ("radon_forward", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    ("radon_backward", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    ("radon_forward_ex", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
      ctypes.POINTER(radon_launch_config), ctypes.c_void_p]),
    ("radon_backward_ex", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
      ctypes.POINTER(radon_launch_config), ctypes.c_void_p]),
    ("radon_forward_workspace_size", ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    ("radon_forward_images_per_cta", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(radon_launch_config), ctypes.POINTER(ctypes.c_int)]),
    ("radon_forward_ws", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
      ctypes.POINTER(radon_launch_config), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("radon_backward_workspace_size", ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    ("radon_backward_ws", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
      ctypes.POINTER(radon_launch_config), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("radon_forward_static_scratch", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    ("radon_forward_fused", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(radon_epilogue),
      ctypes.POINTER(radon_launch_config), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("radon_backward_fused", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(radon_epilogue),
      ctypes.POINTER(radon_launch_config), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("radon_dot_workspace_size", ctypes.c_size_t, []),
    ("radon_dot", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p, ctypes.c_int,
      ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("radon_axpby", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p,
      ctypes.c_float, ctypes.c_void_p]),
    ("radon_power_iteration_workspace_size", ctypes.c_size_t, [ctypes.c_void_p]),
    ("radon_power_iteration", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
      ctypes.c_size_t, ctypes.c_void_p]),
    ("radon_batch_plan_create", ctypes.c_int,
     [ctypes.POINTER(radon_item), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(radon_plan_options),
      ctypes.POINTER(ctypes.c_void_p)]),
    ("radon_batch_plan_launch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("radon_batch_plan_get_info", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(radon_plan_info)]),
    ("radon_batch_plan_item_config", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("radon_batch_plan_item_shape", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    ("radon_batch_plan_item_rows", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("radon_batch_plan_destroy", None, [ctypes.c_void_p]),
    ("radon_probe_gather_ceiling", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    ("radon_probe_gather_ceiling_ex", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    ("radon_probe_gather_ceiling_groups", ctypes.c_int,
     [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    ("radon_filter_sinogram", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    ("radon_dot_batched_workspace_size", ctypes.c_size_t, [ctypes.c_int]),
    ("radon_dot_batched", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p,
      ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("radon_axpby_batched", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_float,
      ctypes.c_void_p, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    ("radon_safe_divide", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("radon_cgne_workspace_size", ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int]),
    ("radon_cgne", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
      ctypes.c_size_t, ctypes.c_void_p]),
    ("radon_backproject_interpolating", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    ("radon_backproject_interpolating_ws", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
      ctypes.c_void_p]),
    ("radon_kernel_launch_count", ctypes.c_uint64, []),
    ("radon_get_device_error", ctypes.c_int, [ctypes.c_void_p]),
    ("radon_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("radon_last_error_message", ctypes.c_char_p, []),
    ("radon_abi_version", ctypes.c_int, []),
]


def load() -> ctypes.CDLL:
    """The loaded library.  Raises if ``libradon.so`` is missing (build it first)."""
    global _c
    if _c is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libradon.so is not built (%s); run paper_2009_14788_gb300.build.build() — "
                               "there is no CPU fallback" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _c = lib
    return _c


def exported_names() -> list[str]:
    return [s[0] for s in _SIGNATURES]


def status_string(status: int) -> str:
    return load().radon_status_string(status).decode()


def radon_last_error_message() -> str:
    return load().radon_last_error_message().decode()


def check(status: int, where: str) -> None:
    if status != RADON_OK:
        raise RadonError(status, where, radon_last_error_message())


def _call(name, *args):
    return getattr(load(), name)(*args)


# Thin same-name wrappers (return the raw status; ``check`` turns it into an exception).
def radon_geometry_create_parallel(n, angles_ptr, n_angles, det_count, det_spacing, step, out_ptr):
    return _call("radon_geometry_create_parallel", n, angles_ptr, n_angles, det_count, det_spacing, step, out_ptr)


def radon_geometry_create_fanbeam(n, angles_ptr, n_angles, source_distance, det_distance, det_count, det_spacing,
                                  step, out_ptr):
    return _call("radon_geometry_create_fanbeam", n, angles_ptr, n_angles, source_distance, det_distance, det_count,
                 det_spacing, step, out_ptr)


def radon_geometry_create(desc, out_ptr):
    return _call("radon_geometry_create", desc, out_ptr)


def radon_geometry_copy_rays(geom, rays_ptr, counts_ptr):
    return _call("radon_geometry_copy_rays", geom, rays_ptr, counts_ptr)


def radon_geometry_destroy(geom):
    return _call("radon_geometry_destroy", geom)


def radon_geometry_get_info(geom, info_ptr):
    return _call("radon_geometry_get_info", geom, info_ptr)


def radon_geometry_sample_count(geom):
    return _call("radon_geometry_sample_count", geom)


def radon_geometry_adjoint_table_size(geom, bytes_ptr):
    return _call("radon_geometry_adjoint_table_size", geom, bytes_ptr)


def radon_geometry_build_adjoint_table(geom):
    return _call("radon_geometry_build_adjoint_table", geom)


def radon_geometry_adjoint_table_overflow(geom, fraction_ptr):
    return _call("radon_geometry_adjoint_table_overflow", geom, fraction_ptr)


def radon_geometry_free_adjoint_table(geom):
    return _call("radon_geometry_free_adjoint_table", geom)


def radon_forward(geom, img, sino, dtype, batch, stream):
    return _call("radon_forward", geom, img, sino, dtype, batch, stream)


def radon_backward(geom, sino, img, dtype, batch, stream):
    return _call("radon_backward", geom, sino, img, dtype, batch, stream)


def radon_forward_ex(geom, img, sino, dtype, batch, config, stream):
    return _call("radon_forward_ex", geom, img, sino, dtype, batch, config, stream)


def radon_backward_ex(geom, sino, img, dtype, batch, config, stream):
    return _call("radon_backward_ex", geom, sino, img, dtype, batch, config, stream)


def radon_forward_workspace_size(geom, dtype, batch):
    return _call("radon_forward_workspace_size", geom, dtype, batch)


def radon_forward_images_per_cta(geom, dtype, batch, config_ptr, images_ptr):
    return _call("radon_forward_images_per_cta", geom, dtype, batch, config_ptr, images_ptr)


def radon_forward_ws(geom, img, sino, dtype, batch, config, workspace, workspace_bytes, stream):
    return _call("radon_forward_ws", geom, img, sino, dtype, batch, config, workspace, workspace_bytes, stream)


def radon_backward_workspace_size(geom, dtype, batch):
    return _call("radon_backward_workspace_size", geom, dtype, batch)


def radon_backward_ws(geom, sino, img, dtype, batch, config, workspace, workspace_bytes, stream):
    return _call("radon_backward_ws", geom, sino, img, dtype, batch, config, workspace, workspace_bytes, stream)


def radon_forward_static_scratch(geom, img, sino, dtype, batch, stream):
    return _call("radon_forward_static_scratch", geom, img, sino, dtype, batch, stream)


def radon_forward_fused(geom, img, sino, dtype, batch, epilogue, config, workspace, workspace_bytes, stream):
    return _call("radon_forward_fused", geom, img, sino, dtype, batch, epilogue, config, workspace, workspace_bytes,
                 stream)


def radon_backward_fused(geom, sino, img, dtype, batch, epilogue, config, workspace, workspace_bytes, stream):
    return _call("radon_backward_fused", geom, sino, img, dtype, batch, epilogue, config, workspace, workspace_bytes,
                 stream)


def radon_dot_workspace_size():
    return _call("radon_dot_workspace_size")


def radon_dot(a, b, dtype, count, scale, result, accumulate, workspace, workspace_bytes, stream):
    return _call("radon_dot", a, b, dtype, count, scale, result, accumulate, workspace, workspace_bytes, stream)


def radon_axpby(x, x_dtype, y, y_dtype, count, alpha, alpha_dev, beta, stream):
    return _call("radon_axpby", x, x_dtype, y, y_dtype, count, alpha, alpha_dev, beta, stream)


def radon_power_iteration_workspace_size(geom):
    return _call("radon_power_iteration_workspace_size", geom)


def radon_power_iteration(geom, v0, iterations, lambda_out, alpha_out, workspace, workspace_bytes, stream):
    return _call("radon_power_iteration", geom, v0, iterations, lambda_out, alpha_out, workspace, workspace_bytes,
                 stream)


def radon_batch_plan_create(items, n, direction, dtype, options, out_ptr):
    return _call("radon_batch_plan_create", items, n, direction, dtype, options, out_ptr)


def radon_batch_plan_launch(plan, stream):
    return _call("radon_batch_plan_launch", plan, stream)


def radon_batch_plan_get_info(plan, info_ptr):
    return _call("radon_batch_plan_get_info", plan, info_ptr)


def radon_batch_plan_item_config(plan, item, views_ptr):
    return _call("radon_batch_plan_item_config", plan, item, views_ptr)


def radon_batch_plan_item_shape(plan, item, views_ptr, lanes_ptr):
    return _call("radon_batch_plan_item_shape", plan, item, views_ptr, lanes_ptr)


def radon_batch_plan_item_rows(plan, item, rows_ptr):
    return _call("radon_batch_plan_item_rows", plan, item, rows_ptr)


def radon_batch_plan_destroy(plan):
    return _call("radon_batch_plan_destroy", plan)


def radon_probe_gather_ceiling(dtype, out_ptr):
    return _call("radon_probe_gather_ceiling", dtype, out_ptr)


def radon_probe_gather_ceiling_ex(dtype, weights, out_ptr):
    return _call("radon_probe_gather_ceiling_ex", dtype, weights, out_ptr)


def radon_probe_gather_ceiling_groups(dtype, weights, groups, out_ptr):
    return _call("radon_probe_gather_ceiling_groups", dtype, weights, groups, out_ptr)


def radon_filter_sinogram(geom, sino, out, dtype, batch, filter_kind, stream):
    return _call("radon_filter_sinogram", geom, sino, out, dtype, batch, filter_kind, stream)


def radon_dot_batched_workspace_size(batch):
    return _call("radon_dot_batched_workspace_size", batch)


def radon_dot_batched(a, b, dtype, batch, count, scale, result, accumulate, workspace, workspace_bytes, stream):
    return _call("radon_dot_batched", a, b, dtype, batch, count, scale, result, accumulate, workspace,
                 workspace_bytes, stream)


def radon_axpby_batched(x, x_dtype, y, y_dtype, batch, count, alpha, alpha_dev, beta, beta_dev, stream):
    return _call("radon_axpby_batched", x, x_dtype, y, y_dtype, batch, count, alpha, alpha_dev, beta, beta_dev, stream)


def radon_safe_divide(num, den, out, batch, stream):
    return _call("radon_safe_divide", num, den, out, batch, stream)


def radon_cgne_workspace_size(geom, batch):
    return _call("radon_cgne_workspace_size", geom, batch)


def radon_cgne(geom, y, x, dtype, batch, iterations, workspace, workspace_bytes, stream):
    return _call("radon_cgne", geom, y, x, dtype, batch, iterations, workspace, workspace_bytes, stream)


def radon_backproject_interpolating(geom, sino, img, dtype, batch, stream):
    return _call("radon_backproject_interpolating", geom, sino, img, dtype, batch, stream)


def radon_backproject_interpolating_ws(geom, sino, img, dtype, batch, workspace, workspace_bytes, stream):
    return _call("radon_backproject_interpolating_ws", geom, sino, img, dtype, batch, workspace, workspace_bytes, stream)


def radon_kernel_launch_count():
    return _call("radon_kernel_launch_count")


def radon_get_device_error(stream):
    return _call("radon_get_device_error", stream)


def radon_abi_version():
    return _call("radon_abi_version")
