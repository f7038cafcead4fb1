"""Conjugate-gradient solvers (Section 2.1's solvers module, used in Section 4.2), every image of a
batch its own problem, every vector operation in libradon's batched kernels.

* ``cgne(radon, x0, y, max_iter)``: CG on the normal equation A^T A x = A^T y (Hanke's CGNE), run
  entirely on the device by ``radon_cgne``.
* ``cg(apply_op, x0, b, max_iter)``: CG for a symmetric positive (semi-)definite operator given as
  a callable on tensors shaped like x0 (e.g. a regularised normal operator built from the projector),
  with per-item step lengths from ``radon_dot_batched`` / ``radon_safe_divide`` /
  ``radon_axpby_batched``.

Both run exactly ``max_iter`` iterations (the paper's solvers take the count under that name;
``iterations=`` is accepted as well); a zero denominator gives a zero step, so a converged problem
stays put.
"""

from __future__ import annotations

import torch

from . import _lib as L
from .radon import _DTYPES, Geometry


def _stream(t: torch.Tensor):
    return torch.cuda.current_stream(t.device).cuda_stream


class _Vec:
    """Per-item vector kernels on tensors with a leading batch axis."""

    def __init__(self, batch: int, device):
        self.batch = batch
        self.ws = torch.empty(max(8, int(L.radon_dot_batched_workspace_size(batch))), dtype=torch.uint8,
                              device=device)

    def dot(self, a, b, out):
        n = a.numel() // self.batch
        L.check(L.radon_dot_batched(a.data_ptr(), b.data_ptr(), _DTYPES[a.dtype], self.batch, n, 1.0, out.data_ptr(),
                                    0, self.ws.data_ptr(), self.ws.numel(), _stream(a)), "radon_dot_batched")
        return out

    def axpby(self, x, y, alpha=1.0, alpha_dev=None, beta=0.0, beta_dev=None):
        n = x.numel() // self.batch
        L.check(L.radon_axpby_batched(x.data_ptr(), _DTYPES[x.dtype], y.data_ptr(), _DTYPES[y.dtype], self.batch, n,
                                      float(alpha), alpha_dev.data_ptr() if alpha_dev is not None else None,
                                      float(beta), beta_dev.data_ptr() if beta_dev is not None else None,
                                      _stream(x)), "radon_axpby_batched")
        return y

    def divide(self, num, den, out):
        L.check(L.radon_safe_divide(num.data_ptr(), den.data_ptr(), out.data_ptr(), self.batch, _stream(num)),
                "radon_safe_divide")
        return out


def _count(max_iter, iterations) -> int:
    if (max_iter is None) == (iterations is None):
        raise ValueError("give the iteration count once, as max_iter (or iterations)")
    n = int(max_iter if max_iter is not None else iterations)
    if n < 0:
        raise ValueError("the iteration count must be >= 0")
    return n


def cgne(radon, x0: torch.Tensor, y: torch.Tensor, max_iter: int | None = None, *,
         iterations: int | None = None) -> torch.Tensor:
    """x_K of CGNE from x0 (``[B, N, N]`` or ``[N, N]``, FP32) for sinograms y (``radon_cgne``)."""
    iterations = _count(max_iter, iterations)
    geom: Geometry = radon.geometry if hasattr(radon, "geometry") else radon
    if x0.dtype != torch.float32 or y.dtype != torch.float32:
        raise ValueError("CGNE runs on FP32 tensors")
    single = x0.dim() == 2
    xb = x0.reshape(-1, geom.n, geom.n)
    yb = y.reshape(-1, *geom.sino_shape).contiguous()
    batch = xb.shape[0]
    if yb.shape[0] != batch:
        raise ValueError("x0 and y hold different batch sizes")
    x = torch.empty(xb.shape, dtype=torch.float32, device=xb.device)
    _Vec(max(batch, 1), x.device).axpby(xb.contiguous(), x, 1.0)   # the start, copied (x0 is kept)
    need = int(L.radon_cgne_workspace_size(geom.handle, max(batch, 1)))
    ws = torch.empty(max(need, 16), dtype=torch.uint8, device=x.device)
    with torch.cuda.device(x.device):
        L.check(L.radon_cgne(geom.handle, yb.data_ptr(), x.data_ptr(), L.RADON_F32, batch, int(iterations),
                             ws.data_ptr(), ws.numel(), _stream(x)), "radon_cgne")
    return x[0] if single else x


def cg(apply_op, x0: torch.Tensor, b: torch.Tensor, max_iter: int | None = None, *,
       iterations: int | None = None) -> torch.Tensor:
    """x_K of CG for apply_op(x) = b: a ``[B, ...]`` tensor holds B problems (one per item along the
    leading axis), a one- or two-dimensional tensor (one image) one problem; apply_op receives and
    returns tensors shaped like x0."""
    iterations = _count(max_iter, iterations)
    if x0.shape != b.shape or x0.dtype != b.dtype:
        raise ValueError("x0 and b must share shape and dtype")
    batch = x0.shape[0] if x0.dim() >= 3 else 1
    v = _Vec(batch, x0.device)
    f32 = dict(dtype=torch.float32, device=x0.device)
    x = v.axpby(x0.contiguous(), torch.empty_like(x0, memory_format=torch.contiguous_format), 1.0)
    r = v.axpby(b.contiguous(), torch.empty_like(x), 1.0)
    v.axpby(apply_op(x).contiguous(), r, -1.0, beta=1.0)          # r = b - M x
    p = v.axpby(r, torch.empty_like(r), 1.0)
    rr, pmp, alpha, beta = (torch.empty(batch, **f32) for _ in range(4))
    rnew = torch.empty(batch, **f32)
    v.dot(r, r, rr)
    for _ in range(int(iterations)):
        mp = apply_op(p).contiguous()
        v.dot(p, mp, pmp)
        v.divide(rr, pmp, alpha)
        v.axpby(p, x, 1.0, alpha_dev=alpha, beta=1.0)                # x += alpha p
        v.axpby(mp, r, -1.0, alpha_dev=alpha, beta=1.0)              # r -= alpha M p
        v.dot(r, r, rnew)
        v.divide(rnew, rr, beta)
        v.axpby(r, p, 1.0, beta=1.0, beta_dev=beta)                  # p = r + beta p
        rr, rnew = rnew, rr
    return x
