"""PyTorch-facing operators over libradon: geometry objects, forward / backprojection, autograd.

The API mirrors the paper's (Section 3.1.1, 3.1.2): ``Radon(resolution, angles, det_count=...)``
and ``RadonFanbeam(resolution, angles, source_distance, det_distance=..., det_count=...,
det_spacing=...)`` with ``.forward(x)`` and ``.backprojection(sino)`` (alias ``.backward``).
Both operators are differentiable (Section 2): the gradient of the forward projection is the
backprojection kernel and vice versa.  PyTorch supplies device memory and the current CUDA
stream; every step of the computation runs in libradon's kernels.
"""

from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L

_DTYPES = {torch.float32: L.RADON_F32, torch.float16: L.RADON_F16, torch.bfloat16: L.RADON_BF16}

ALGOS = {"auto": L.RADON_ALGO_AUTO, "plain": L.RADON_ALGO_PLAIN, "tiled": L.RADON_ALGO_TILED}


def launch_config(algo="auto", views_per_cta=0, rows_per_slab=0, images_per_cta=0, tile=0, threads=0, weights=0):
    """A ``radon_launch_config`` (kernel family and tile parameters; 0 = library default).

    ``weights``: 0 / 1 keep FP32 bilinear weights (the default, single-precision arithmetic in every
    storage type); 2 rounds them to FP16 inside exact mixed-precision products in the FP16 forward
    (opt-in, see include/radon.h)."""
    return L.radon_launch_config(ALGOS[algo] if isinstance(algo, str) else int(algo), views_per_cta, rows_per_slab,
                                 images_per_cta, tile, threads, weights)


class Geometry:
    """Owns a ``radon_geometry*`` (FP64-built tables on one device, or host-only tables)."""

    def __init__(self, kind: str, n: int, angles, det_count=None, det_spacing=None, step=None,
                 source_distance: float = 0.0, det_distance=None, host_only: bool = False, device=None):
        if kind not in ("parallel", "fan"):
            raise ValueError("kind must be 'parallel' or 'fan'")
        self._h = None
        ang = np.ascontiguousarray(np.asarray(angles, dtype=np.float64).reshape(-1))
        self._angles = ang
        desc = L.radon_geometry_desc(
            int(n), ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(ang.size), 1 if kind == "fan" else 0,
            float(source_distance or 0.0), float(det_distance or 0.0), int(det_count or 0),
            float(det_spacing or 0.0), float(step or 0.0), 1 if host_only else 0)
        handle = ctypes.c_void_p()
        if host_only:
            st = L.radon_geometry_create(ctypes.byref(desc), ctypes.byref(handle))
        else:
            dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
            with torch.cuda.device(dev):
                st = L.radon_geometry_create(ctypes.byref(desc), ctypes.byref(handle))
        L.check(st, "radon_geometry_create")
        self._h = handle
        self._lib = L.load()
        info = L.radon_geometry_info()
        L.check(L.radon_geometry_get_info(self._h, ctypes.byref(info)), "radon_geometry_get_info")
        self.kind = kind
        self.host_only = bool(host_only)
        self.n = info.n
        self.n_angles = info.n_angles
        self.det_count = info.det_count
        self.det_spacing = info.det_spacing
        self.step = info.step
        self.source_distance = info.source_distance
        self.det_distance = info.det_distance
        self.sample_count = int(info.sample_count)
        self.device = None if host_only else torch.device("cuda", info.device)

    @property
    def handle(self):
        return self._h

    @property
    def angles(self) -> np.ndarray:
        return self._angles.copy()

    @property
    def sino_shape(self) -> tuple[int, int]:
        return (self.n_angles, self.det_count)

    def rays(self) -> tuple[np.ndarray, np.ndarray]:
        """The split-precision ray table the kernels read: ([V, D, 8] (J0, I0, fx0, fy0, dxh, dyh, dxl, dyl),
        [V, D] sample counts); sample k sits at (J0 + fx0 + k (dxh + dxl), I0 + fy0 + k (dyh + dyl))."""
        rays = np.zeros((self.n_angles, self.det_count, 8), dtype=np.float32)
        counts = np.zeros((self.n_angles, self.det_count), dtype=np.int32)
        L.check(L.radon_geometry_copy_rays(self._h, rays.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                           counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
                "radon_geometry_copy_rays")
        return rays, counts

    def adjoint_table_bytes(self) -> int:
        """Device bytes of the exact adjoint's weight table (see ``build_adjoint_table``)."""
        b = ctypes.c_size_t()
        L.check(L.radon_geometry_adjoint_table_size(self._h, ctypes.byref(b)), "radon_geometry_adjoint_table_size")
        return int(b.value)

    def build_adjoint_table(self) -> None:
        """Precomputes the exact adjoint's bilinear weights on the geometry's device (tiles x views x 128
        pixel pairs x 44 bytes, ``adjoint_table_bytes``); the packed adjoint then reads them instead of
        computing them, with the same bits (pixel pairs whose weighted rays span more than five detectors
        in a view keep computing theirs: ``adjoint_table_overflow``).  Raises ``RadonError``
        (RADON_ERR_UNSUPPORTED) where the packed adjoint cannot serve the geometry."""
        with torch.cuda.device(self.device):
            L.check(L.radon_geometry_build_adjoint_table(self._h), "radon_geometry_build_adjoint_table")

    def adjoint_table_overflow(self) -> float:
        """Fraction of the table's (pixel pair, view) records left to the on-the-fly weights."""
        f = ctypes.c_double()
        L.check(L.radon_geometry_adjoint_table_overflow(self._h, ctypes.byref(f)),
                "radon_geometry_adjoint_table_overflow")
        return float(f.value)

    def free_adjoint_table(self) -> None:
        L.check(L.radon_geometry_free_adjoint_table(self._h), "radon_geometry_free_adjoint_table")

    def close(self):
        if self._h is not None and self._h.value:
            self._lib.radon_geometry_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_tensor(t: torch.Tensor, what: str, geom: Geometry):
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % what)
    if t.device.type != "cuda":
        raise ValueError("%s must be a CUDA tensor (libradon has no CPU path)" % what)
    if geom.device is None:
        raise ValueError("geometry is host-only")
    if t.device != geom.device:
        raise ValueError("%s is on %s but the geometry lives on %s" % (what, t.device, geom.device))
    if t.dtype not in _DTYPES:
        raise TypeError("%s dtype must be float32, float16 or bfloat16, got %s" % (what, t.dtype))


def _check_out(out: torch.Tensor, like: torch.Tensor, shape) -> torch.Tensor:
    """The library writes through raw pointers: an output buffer must match exactly."""
    if not isinstance(out, torch.Tensor):
        raise TypeError("out must be a torch.Tensor")
    if out.dtype != like.dtype or out.device != like.device or tuple(out.shape) != tuple(shape) \
            or not out.is_contiguous():
        raise ValueError("out must be a contiguous %s tensor of shape %s on %s, got %s %s on %s"
                         % (like.dtype, tuple(shape), like.device, out.dtype, tuple(out.shape), out.device))
    return out


def forward_workspace_bytes(geom: Geometry, dtype: torch.dtype, batch: int) -> int:
    """Bytes of the workspace the packed forward path uses (``radon_forward_workspace_size``)."""
    return int(L.radon_forward_workspace_size(geom.handle, _DTYPES[dtype], int(batch)))


def forward_images_per_cta(geom: Geometry, dtype: torch.dtype, batch: int, config=None) -> int:
    """Images per CTA of the packed forward for this call (``radon_forward_images_per_cta``): one texel
    group (8 for 16-bit storage, 4 for FP32) or two; 0 when another kernel serves it."""
    n = ctypes.c_int(0)
    L.check(L.radon_forward_images_per_cta(geom.handle, _DTYPES[dtype], int(batch),
                                           ctypes.byref(config) if config is not None else None, ctypes.byref(n)),
            "radon_forward_images_per_cta")
    return int(n.value)


def forward_raw(geom: Geometry, x: torch.Tensor, config=None, out=None, workspace="auto") -> torch.Tensor:
    """y = A x through the C ABI (no autograd).

    ``workspace``: "auto" allocates the packed-path workspace from PyTorch's caching allocator on
    the current stream; a uint8 CUDA tensor is used as given; None runs the paths that need none.
    """
    _check_tensor(x, "image", geom)
    if x.shape[-2:] != (geom.n, geom.n):
        raise ValueError("image must end in (%d, %d), got %s" % (geom.n, geom.n, tuple(x.shape)))
    x = x.contiguous()
    batch = x.numel() // (geom.n * geom.n)
    shape = tuple(x.shape[:-2]) + geom.sino_shape
    y = torch.empty(shape, dtype=x.dtype, device=x.device) if out is None else _check_out(out, x, shape)
    stream = torch.cuda.current_stream(x.device).cuda_stream
    ws_ptr, ws_bytes = None, 0
    if isinstance(workspace, str) and workspace == "auto":
        need = forward_workspace_bytes(geom, x.dtype, batch)
        if need > 0 and batch > 0:
            workspace = torch.empty(need, dtype=torch.uint8, device=x.device)
        else:
            workspace = None
    if isinstance(workspace, torch.Tensor):
        if workspace.device != x.device or not workspace.is_contiguous():
            raise ValueError("workspace must be a contiguous tensor on %s" % x.device)
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    with torch.cuda.device(x.device):
        cfg = ctypes.byref(config) if config is not None else None
        if ws_ptr is not None:
            st = L.radon_forward_ws(geom.handle, x.data_ptr(), y.data_ptr(), _DTYPES[x.dtype], batch, cfg, ws_ptr,
                                    ws_bytes, stream)
        elif config is None:
            st = L.radon_forward(geom.handle, x.data_ptr(), y.data_ptr(), _DTYPES[x.dtype], batch, stream)
        else:
            st = L.radon_forward_ex(geom.handle, x.data_ptr(), y.data_ptr(), _DTYPES[x.dtype], batch, cfg, stream)
    L.check(st, "radon_forward")
    return y


def backward_workspace_bytes(geom: Geometry, dtype: torch.dtype, batch: int) -> int:
    """Bytes of the workspace the packed adjoint path uses (``radon_backward_workspace_size``)."""
    return int(L.radon_backward_workspace_size(geom.handle, _DTYPES[dtype], int(batch)))


def _workspace(workspace, need, device):
    if isinstance(workspace, str) and workspace == "auto":
        return torch.empty(need, dtype=torch.uint8, device=device) if need > 0 else None
    if isinstance(workspace, torch.Tensor):
        if workspace.device != device or not workspace.is_contiguous():
            raise ValueError("workspace must be a contiguous tensor on %s" % device)
        return workspace
    return None


def backward_raw(geom: Geometry, y: torch.Tensor, config=None, out=None, workspace="auto") -> torch.Tensor:
    """x = A^T y through the C ABI (no autograd); ``workspace`` as for ``forward_raw``."""
    _check_tensor(y, "sinogram", geom)
    if tuple(y.shape[-2:]) != geom.sino_shape:
        raise ValueError("sinogram must end in %s, got %s" % (geom.sino_shape, tuple(y.shape)))
    y = y.contiguous()
    batch = y.numel() // (geom.n_angles * geom.det_count)
    shape = tuple(y.shape[:-2]) + (geom.n, geom.n)
    x = torch.empty(shape, dtype=y.dtype, device=y.device) if out is None else _check_out(out, y, shape)
    stream = torch.cuda.current_stream(y.device).cuda_stream
    ws = _workspace(workspace, backward_workspace_bytes(geom, y.dtype, batch) if batch > 0 else 0, y.device)
    with torch.cuda.device(y.device):
        cfg = ctypes.byref(config) if config is not None else None
        if ws is not None:
            st = L.radon_backward_ws(geom.handle, y.data_ptr(), x.data_ptr(), _DTYPES[y.dtype], batch, cfg,
                                     ws.data_ptr(), ws.numel() * ws.element_size(), stream)
        elif config is None:
            st = L.radon_backward(geom.handle, y.data_ptr(), x.data_ptr(), _DTYPES[y.dtype], batch, stream)
        else:
            st = L.radon_backward_ex(geom.handle, y.data_ptr(), x.data_ptr(), _DTYPES[y.dtype], batch, cfg, stream)
    L.check(st, "radon_backward")
    return x


def _epilogue(op_scale, op_scale_dev, add_scale, add, like: torch.Tensor):
    if op_scale_dev is not None:
        if op_scale_dev.dtype != torch.float32 or op_scale_dev.device != like.device or op_scale_dev.numel() != 1:
            raise ValueError("op_scale_dev must be one float32 element on %s" % like.device)
    if add is not None:
        if add.dtype != like.dtype or add.device != like.device or not add.is_contiguous():
            raise ValueError("add must be a contiguous %s tensor on %s" % (like.dtype, like.device))
    return L.radon_epilogue(float(op_scale), op_scale_dev.data_ptr() if op_scale_dev is not None else None,
                            float(add_scale), add.data_ptr() if add is not None else None)


def forward_fused(geom: Geometry, x: torch.Tensor, op_scale=1.0, op_scale_dev=None, add=None, add_scale=0.0,
                  out=None, config=None, workspace="auto") -> torch.Tensor:
    """out = op_scale * s * (A x) + add_scale * add, s = op_scale_dev[0] (``radon_forward_fused``).

    ``add`` (the sinogram's shape and dtype) may be ``out`` itself; the sum is rounded once.
    """
    _check_tensor(x, "image", geom)
    x = x.contiguous()
    batch = x.numel() // (geom.n * geom.n)
    shape = tuple(x.shape[:-2]) + geom.sino_shape
    y = torch.empty(shape, dtype=x.dtype, device=x.device) if out is None else _check_out(out, x, shape)
    if add is not None and tuple(add.shape) != shape:
        raise ValueError("add must have shape %s" % (shape,))
    ep = _epilogue(op_scale, op_scale_dev, add_scale, add, y)
    ws = _workspace(workspace, forward_workspace_bytes(geom, x.dtype, batch) if batch > 0 else 0, x.device)
    stream = torch.cuda.current_stream(x.device).cuda_stream
    with torch.cuda.device(x.device):
        st = L.radon_forward_fused(geom.handle, x.data_ptr(), y.data_ptr(), _DTYPES[x.dtype], batch, ctypes.byref(ep),
                                   ctypes.byref(config) if config is not None else None,
                                   ws.data_ptr() if ws is not None else None,
                                   ws.numel() if ws is not None else 0, stream)
    L.check(st, "radon_forward_fused")
    return y


def backward_fused(geom: Geometry, y: torch.Tensor, op_scale=1.0, op_scale_dev=None, add=None, add_scale=0.0,
                   out=None, config=None, workspace="auto") -> torch.Tensor:
    """out = op_scale * s * (A^T y) + add_scale * add, s = op_scale_dev[0] (``radon_backward_fused``)."""
    _check_tensor(y, "sinogram", geom)
    if tuple(y.shape[-2:]) != geom.sino_shape:
        raise ValueError("sinogram must end in %s, got %s" % (geom.sino_shape, tuple(y.shape)))
    y = y.contiguous()
    batch = y.numel() // (geom.n_angles * geom.det_count)
    shape = tuple(y.shape[:-2]) + (geom.n, geom.n)
    x = torch.empty(shape, dtype=y.dtype, device=y.device) if out is None else _check_out(out, y, shape)
    if add is not None and tuple(add.shape) != shape:
        raise ValueError("add must have shape %s" % (shape,))
    ep = _epilogue(op_scale, op_scale_dev, add_scale, add, x)
    ws = _workspace(workspace, backward_workspace_bytes(geom, y.dtype, batch) if batch > 0 else 0, y.device)
    stream = torch.cuda.current_stream(y.device).cuda_stream
    with torch.cuda.device(y.device):
        st = L.radon_backward_fused(geom.handle, y.data_ptr(), x.data_ptr(), _DTYPES[y.dtype], batch, ctypes.byref(ep),
                                    ctypes.byref(config) if config is not None else None,
                                    ws.data_ptr() if ws is not None else None,
                                    ws.numel() if ws is not None else 0, stream)
    L.check(st, "radon_backward_fused")
    return x


def dot(a: torch.Tensor, b: torch.Tensor, result=None, scale=1.0, accumulate=False, workspace=None) -> torch.Tensor:
    """result = scale * <a, b> (+ result if ``accumulate``) as one device float32 (``radon_dot``)."""
    if a.dtype != b.dtype or a.numel() != b.numel() or a.device != b.device:
        raise ValueError("a and b must have the same dtype, size and device")
    if a.dtype not in _DTYPES:
        raise ValueError("unsupported dtype %s" % a.dtype)
    a, b = a.contiguous(), b.contiguous()
    if result is None:
        result = torch.empty(1, dtype=torch.float32, device=a.device)
    need = int(L.radon_dot_workspace_size())
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=a.device)
    stream = torch.cuda.current_stream(a.device).cuda_stream
    with torch.cuda.device(a.device):
        st = L.radon_dot(a.data_ptr(), b.data_ptr(), _DTYPES[a.dtype], a.numel(), float(scale), result.data_ptr(),
                         1 if accumulate else 0, workspace.data_ptr(), workspace.numel(), stream)
    L.check(st, "radon_dot")
    return result


def axpby(x: torch.Tensor, y: torch.Tensor, alpha=1.0, alpha_dev=None, beta=0.0) -> torch.Tensor:
    """y = alpha * s * x + beta * y in place (s = alpha_dev[0]); x and y may differ in dtype (``radon_axpby``)."""
    if x.numel() != y.numel() or x.device != y.device or not x.is_contiguous() or not y.is_contiguous():
        raise ValueError("x and y must be contiguous tensors of the same size on one device")
    if alpha_dev is not None and (alpha_dev.dtype != torch.float32 or alpha_dev.device != x.device):
        raise ValueError("alpha_dev must be a float32 tensor on %s" % x.device)
    stream = torch.cuda.current_stream(x.device).cuda_stream
    with torch.cuda.device(x.device):
        st = L.radon_axpby(x.data_ptr(), _DTYPES[x.dtype], y.data_ptr(), _DTYPES[y.dtype], x.numel(), float(alpha),
                           alpha_dev.data_ptr() if alpha_dev is not None else None, float(beta), stream)
    L.check(st, "radon_axpby")
    return y


def power_iteration(geom: Geometry, v0: torch.Tensor, iterations: int = 20):
    """(lambda, alpha = 1 / lambda) of A^T A by the power method from ``v0`` (``radon_power_iteration``).

    Both are one-element float32 device tensors; nothing is synchronised.
    """
    if v0.dtype != torch.float32 or v0.numel() != geom.n * geom.n or not v0.is_cuda:
        raise ValueError("v0 must be one float32 %dx%d image on the GPU" % (geom.n, geom.n))
    v0 = v0.contiguous()
    lam = torch.empty(1, dtype=torch.float32, device=v0.device)
    alpha = torch.empty(1, dtype=torch.float32, device=v0.device)
    need = int(L.radon_power_iteration_workspace_size(geom.handle))
    ws = torch.empty(need, dtype=torch.uint8, device=v0.device)
    stream = torch.cuda.current_stream(v0.device).cuda_stream
    with torch.cuda.device(v0.device):
        st = L.radon_power_iteration(geom.handle, v0.data_ptr(), int(iterations), lam.data_ptr(), alpha.data_ptr(),
                                     ws.data_ptr(), need, stream)
    L.check(st, "radon_power_iteration")
    return lam, alpha


def backproject_interpolating(geom: Geometry, y: torch.Tensor, out=None, workspace="auto") -> torch.Tensor:
    """Pixel-driven interpolating backprojection (``radon_backproject_interpolating[_ws]``):
    approximates the exact adjoint, cheaper; not differentiable (it is not the forward's transpose).
    ``workspace`` as for ``backward_raw`` ("auto": the packed TMA pipeline; None: the plain kernel)."""
    _check_tensor(y, "sinogram", geom)
    if tuple(y.shape[-2:]) != geom.sino_shape:
        raise ValueError("sinogram must end in %s, got %s" % (geom.sino_shape, tuple(y.shape)))
    y = y.contiguous()
    batch = y.numel() // (geom.n_angles * geom.det_count)
    shape = tuple(y.shape[:-2]) + (geom.n, geom.n)
    x = torch.empty(shape, dtype=y.dtype, device=y.device) if out is None else _check_out(out, y, shape)
    ws = _workspace(workspace, backward_workspace_bytes(geom, y.dtype, batch) if batch > 0 else 0, y.device)
    stream = torch.cuda.current_stream(y.device).cuda_stream
    with torch.cuda.device(y.device):
        if ws is not None:
            st = L.radon_backproject_interpolating_ws(geom.handle, y.data_ptr(), x.data_ptr(), _DTYPES[y.dtype], batch,
                                                      ws.data_ptr(), ws.numel() * ws.element_size(), stream)
        else:
            st = L.radon_backproject_interpolating(geom.handle, y.data_ptr(), x.data_ptr(), _DTYPES[y.dtype], batch,
                                                   stream)
    L.check(st, "radon_backproject_interpolating")
    return x


def filter_sinogram(geom: Geometry, y: torch.Tensor, filter_name: str = "ram-lak", out=None) -> torch.Tensor:
    """Each view filtered along the detector for FBP (``radon_filter_sinogram``; no autograd)."""
    if filter_name not in L.FILTERS:
        raise ValueError("filter must be one of %s" % ", ".join(L.FILTERS))
    _check_tensor(y, "sinogram", geom)
    if tuple(y.shape[-2:]) != geom.sino_shape:
        raise ValueError("sinogram must end in %s, got %s" % (geom.sino_shape, tuple(y.shape)))
    y = y.contiguous()
    batch = y.numel() // (geom.n_angles * geom.det_count)
    q = torch.empty_like(y) if out is None else _check_out(out, y, tuple(y.shape))
    stream = torch.cuda.current_stream(y.device).cuda_stream
    with torch.cuda.device(y.device):
        st = L.radon_filter_sinogram(geom.handle, y.data_ptr(), q.data_ptr(), _DTYPES[y.dtype], batch,
                                     L.FILTERS[filter_name], stream)
    L.check(st, "radon_filter_sinogram")
    return q


class FilterSinogramFunction(torch.autograd.Function):
    """q = F y with F the (symmetric Toeplitz) FBP filter: dL/dy = F dL/dq."""

    @staticmethod
    def forward(ctx, y, geom, filter_name):
        ctx.geom, ctx.filter_name = geom, filter_name
        return filter_sinogram(geom, y, filter_name)

    @staticmethod
    def backward(ctx, grad):
        return filter_sinogram(ctx.geom, grad.contiguous(), ctx.filter_name), None, None


class BatchPlan:
    """One persistent launch over an uneven batch (``radon_batch_plan_*``).

    ``items``: a list of ``(geometry, input, output)``; inputs are image batches ``[B, N, N]`` (or
    ``[N, N]``) for ``direction="forward"`` and sinograms ``[B, V, D]`` for ``"adjoint"``, outputs
    the matching results, all contiguous CUDA tensors of one dtype on one device.  The plan keeps
    references to the tensors (their addresses are baked in) and writes the outputs at every
    ``launch()``; creation autotunes the shapes per image size unless ``autotune=False`` or the
    shapes are given (forward: ``forward_views``, ``forward_lanes`` and, for the staged kernel,
    ``forward_rows``; adjoint: ``adjoint_views``).  ``forward_kernel``: ``"auto"`` (the staged kernel
    where its bands fit shared memory, else the L1 gather), ``"staged"`` or ``"gather"``.
    ``RADON_TUNE_CACHE`` names a file that keeps the picks across plans.  ``launch()`` is capturable
    in a CUDA graph.
    """

    def __init__(self, items, direction="forward", autotune=True, forward_views=0, adjoint_views=0, forward_lanes=0,
                 forward_rows=0, forward_kernel="auto"):
        if direction not in ("forward", "adjoint"):
            raise ValueError("direction must be 'forward' or 'adjoint'")
        self._h = None
        self.direction = direction
        self._keep = []
        arr = (L.radon_item * max(1, len(items)))()
        dtype = None
        device = None
        for k, (geom, inp, out) in enumerate(items):
            if direction == "forward":
                ishape, oshape = (geom.n, geom.n), geom.sino_shape
            else:
                ishape, oshape = geom.sino_shape, (geom.n, geom.n)
            for t, shp, what in ((inp, ishape, "input"), (out, oshape, "output")):
                if not t.is_cuda or not t.is_contiguous() or tuple(t.shape[-2:]) != tuple(shp):
                    raise ValueError("item %d: %s must be a contiguous CUDA tensor ending in %s" % (k, what, shp))
            if inp.numel() // (ishape[0] * ishape[1]) != out.numel() // (oshape[0] * oshape[1]):
                raise ValueError("item %d: input and output batch sizes differ" % k)
            dtype = inp.dtype if dtype is None else dtype
            device = inp.device if device is None else device
            if inp.dtype != dtype or out.dtype != dtype or inp.device != device or out.device != device:
                raise ValueError("item %d: every tensor must share one dtype and device" % k)
            arr[k] = L.radon_item(geom.handle, inp.data_ptr(), out.data_ptr(), inp.numel() // (ishape[0] * ishape[1]))
            self._keep += [geom, inp, out]
        self.dtype = dtype if dtype is not None else torch.float32
        kernels = {"auto": 0, "staged": 1, "gather": -1}
        if forward_kernel not in kernels:
            raise ValueError("forward_kernel must be 'auto', 'staged' or 'gather'")
        opts = L.radon_plan_options(1 if autotune else 0, int(forward_views), int(adjoint_views), int(forward_lanes),
                                    int(forward_rows), kernels[forward_kernel])
        h = ctypes.c_void_p()
        with torch.cuda.device(device if device is not None else torch.cuda.current_device()):
            st = L.radon_batch_plan_create(arr, len(items), 0 if direction == "forward" else 1, _DTYPES[self.dtype],
                                           ctypes.byref(opts), ctypes.byref(h))
        L.check(st, "radon_batch_plan_create")
        self._h = h
        self._lib = L.load()
        self.device = device
        self.n_items = len(items)

    def launch(self):
        stream = torch.cuda.current_stream(self.device).cuda_stream if self.device is not None else None
        L.check(L.radon_batch_plan_launch(self._h, stream), "radon_batch_plan_launch")

    @property
    def info(self) -> dict:
        inf = L.radon_plan_info()
        L.check(L.radon_batch_plan_get_info(self._h, ctypes.byref(inf)), "radon_batch_plan_get_info")
        return {"units": inf.units, "work_items": inf.work_items, "ctas": inf.ctas,
                "direction": "forward" if inf.direction == 0 else "adjoint"}

    def item_config(self, item: int) -> int:
        v = ctypes.c_int()
        L.check(L.radon_batch_plan_item_config(self._h, int(item), ctypes.byref(v)), "radon_batch_plan_item_config")
        return v.value

    def item_shape(self, item: int) -> tuple[int, int]:
        """(views per forward ray block or adjoint chunk, lanes per forward ray) of item ``item``."""
        v, l = ctypes.c_int(), ctypes.c_int()
        L.check(L.radon_batch_plan_item_shape(self._h, int(item), ctypes.byref(v), ctypes.byref(l)),
                "radon_batch_plan_item_shape")
        return v.value, l.value

    def item_rows(self, item: int) -> int:
        """Texel rows per slab of item ``item`` (staged forward; 0 for the L1 gather and the adjoint)."""
        r = ctypes.c_int()
        L.check(L.radon_batch_plan_item_rows(self._h, int(item), ctypes.byref(r)), "radon_batch_plan_item_rows")
        return r.value

    def close(self):
        if self._h is not None:
            self._lib.radon_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RadonForwardFunction(torch.autograd.Function):
    """y = A x; dL/dx = A^T dL/dy (the adjoint kernel)."""

    @staticmethod
    def forward(ctx, x, geom, config):
        ctx.geom = geom
        ctx.config = config
        return forward_raw(geom, x, config)

    @staticmethod
    def backward(ctx, grad):
        return backward_raw(ctx.geom, grad.contiguous(), ctx.config), None, None


class RadonBackprojectionFunction(torch.autograd.Function):
    """x = A^T y; dL/dy = A dL/dx (the forward kernel)."""

    @staticmethod
    def forward(ctx, y, geom, config):
        ctx.geom = geom
        ctx.config = config
        return backward_raw(geom, y, config)

    @staticmethod
    def backward(ctx, grad):
        return forward_raw(ctx.geom, grad.contiguous(), ctx.config), None, None


class _CastFunction(torch.autograd.Function):
    """A differentiable dtype cast through ``radon_axpby`` (forward to ``dtype``, gradient back)."""

    @staticmethod
    def forward(ctx, x, dtype):
        ctx.src = x.dtype
        out = torch.empty(x.shape, dtype=dtype, device=x.device)
        return axpby(x.contiguous(), out, 1.0, beta=0.0)

    @staticmethod
    def backward(ctx, grad):
        out = torch.empty(grad.shape, dtype=ctx.src, device=grad.device)
        return axpby(grad.contiguous(), out, 1.0, beta=0.0), None


def _autocast(t: torch.Tensor) -> torch.Tensor:
    """Under ``torch.autocast("cuda", dtype=float16 | bfloat16)`` an FP32 input takes the autocast type,
    so the operators run their 16-bit storage paths without the caller changing dtypes (the paper's
    transparent half precision, Section 2); outside autocast, or for other types, it passes as is."""
    if t.dtype == torch.float32 and t.is_cuda and torch.is_autocast_enabled("cuda"):
        dt = torch.get_autocast_dtype("cuda")
        if dt in (torch.float16, torch.bfloat16):
            return _CastFunction.apply(t, dt)
    return t


class Radon:
    """Parallel-beam projector (Section 3.1.1): ``Radon(resolution, angles, det_count=None, det_spacing=1.0)``."""

    def __init__(self, resolution: int, angles, det_count=None, det_spacing=None, step=None, device=None,
                 config=None):
        self.geometry = Geometry("parallel", resolution, angles, det_count, det_spacing, step, device=device)
        self.config = config

    @property
    def resolution(self) -> int:
        return self.geometry.n

    @property
    def sample_count(self) -> int:
        return self.geometry.sample_count

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        return RadonForwardFunction.apply(_autocast(x), self.geometry, self.config)

    def backprojection(self, sino: torch.Tensor) -> torch.Tensor:
        return RadonBackprojectionFunction.apply(_autocast(sino), self.geometry, self.config)

    backward = backprojection

    def build_adjoint_table(self) -> None:
        """Precomputes the exact adjoint's weights for this geometry (``Geometry.build_adjoint_table``):
        batched backprojections then read them, with the same bits."""
        self.geometry.build_adjoint_table()

    def filter_sinogram(self, sino: torch.Tensor, filter_name: str = "ram-lak") -> torch.Tensor:
        """Section 3.1.3: the sinogram filtered for filtered backprojection (differentiable)."""
        return FilterSinogramFunction.apply(_autocast(sino), self.geometry, filter_name)

    def backprojection_interpolating(self, sino: torch.Tensor) -> torch.Tensor:
        """Pixel-driven interpolating backprojection (approximates ``backprojection``; no autograd)."""
        return backproject_interpolating(self.geometry, _autocast(sino))

    def fbp(self, sino: torch.Tensor, filter_name: str = "ram-lak") -> torch.Tensor:
        """Filtered backprojection: ``backprojection(filter_sinogram(sino))`` (parallel beam)."""
        return self.backprojection(self.filter_sinogram(sino, filter_name))

    __call__ = forward


class RadonFanbeam(Radon):
    """Fan-beam projector with a flat detector (Section 3.1.2)."""

    def __init__(self, resolution: int, angles, source_distance: float, det_distance=None, det_count=None,
                 det_spacing=None, step=None, device=None, config=None):
        self.geometry = Geometry("fan", resolution, angles, det_count, det_spacing, step,
                                 source_distance=source_distance, det_distance=det_distance, device=device)
        self.config = config
