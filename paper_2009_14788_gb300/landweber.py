"""Landweber iteration (Section 4.2) on libradon's fused kernels, differentiable w.r.t. y and alpha.

    x_{k+1} = x_k - alpha A^T (A x_k - y),   alpha = 1 / lambda_max(A^T A) from the power method.

Every arithmetic step runs in libradon: the residual r_k = A x_k - y is one forward projection
whose epilogue subtracts y before the single rounding to the storage type, and the update is one
adjoint whose epilogue forms x_k - alpha A^T r_k (alpha stays a device scalar throughout).

Reverse mode with per-iteration checkpointing: the forward pass keeps only the iterates x_k; the
backward pass recomputes each residual and runs, for k = K-1 .. 0 (g_K = dL/dx_K),
    t = A g_{k+1};   dL/dalpha -= <t, r_k>   (= <g_{k+1}, A^T r_k>, the adjoint identity);
    dL/dy += alpha t;   g_k = g_{k+1} - alpha A^T t,
and dL/dx_0 = g_0.  Each backward step is three projections, one inner product and one scaled add.
"""

from __future__ import annotations

import numpy as np
import torch

from . import _lib as L
from .radon import (Geometry, axpby, backward_fused, backward_workspace_bytes, dot, forward_fused,
                    forward_workspace_bytes, power_iteration)


class _Buffers:
    """Workspaces reused by every projection of one Landweber pass."""

    def __init__(self, geom: Geometry, dtype: torch.dtype, batch: int, device):
        fb = forward_workspace_bytes(geom, dtype, batch)
        bb = backward_workspace_bytes(geom, dtype, batch)
        self.fws = torch.empty(max(fb, 16), dtype=torch.uint8, device=device)
        self.bws = torch.empty(max(bb, 16), dtype=torch.uint8, device=device)
        self.dws = torch.empty(int(L.radon_dot_workspace_size()), dtype=torch.uint8, device=device)

    def fwd(self, geom, x, **kw):
        return forward_fused(geom, x, workspace=self.fws, **kw)

    def adj(self, geom, y, **kw):
        return backward_fused(geom, y, workspace=self.bws, **kw)


def _alpha_tensor(alpha, device) -> torch.Tensor:
    if isinstance(alpha, torch.Tensor):
        if alpha.numel() != 1 or alpha.dtype != torch.float32 or alpha.device != device:
            raise ValueError("alpha must be one float32 element on %s" % device)
        return alpha.reshape(1).contiguous()
    return torch.full((1,), float(alpha), dtype=torch.float32, device=device)


class LandweberFunction(torch.autograd.Function):
    """x_K of K Landweber steps from x_0; gradients w.r.t. y, alpha and x_0."""

    @staticmethod
    def forward(ctx, y, alpha, x0, geom, iterations, config):
        if iterations < 0:
            raise ValueError("iterations must be >= 0")
        y = y.contiguous()
        batch = y.numel() // (geom.n_angles * geom.det_count)
        bufs = _Buffers(geom, y.dtype, batch, y.device)
        a = alpha.reshape(1).contiguous()
        xs = [x0.contiguous()]
        if iterations == 0:
            xs.append(axpby(xs[0], torch.empty_like(xs[0]), 1.0, beta=0.0))   # a fresh output, not x0
        r = torch.empty_like(y)
        for _ in range(iterations):
            bufs.fwd(geom, xs[-1], add=y, add_scale=-1.0, out=r, config=config)                  # r = A x - y
            xs.append(bufs.adj(geom, r, op_scale=-1.0, op_scale_dev=a, add=xs[-1], add_scale=1.0,
                               config=config))                                                     # x - alpha A^T r
        ctx.geom, ctx.iterations, ctx.config = geom, iterations, config
        ctx.save_for_backward(y, a, *xs[:-1])
        return xs[-1]

    @staticmethod
    def backward(ctx, grad):
        geom, K, config = ctx.geom, ctx.iterations, ctx.config
        y, a, *xs = ctx.saved_tensors
        batch = y.numel() // (geom.n_angles * geom.det_count)
        bufs = _Buffers(geom, y.dtype, batch, y.device)
        g = torch.empty_like(xs[0] if xs else grad)
        axpby(grad.contiguous(), g, 1.0, beta=0.0)            # g_K (a private copy, updated in place)
        dalpha = torch.zeros(1, dtype=torch.float32, device=y.device) if K == 0 else \
            torch.empty(1, dtype=torch.float32, device=y.device)
        dy32 = torch.empty(y.shape, dtype=torch.float32, device=y.device)
        if K == 0:
            axpby(y, dy32, 0.0, beta=0.0)
        r = torch.empty_like(y)
        t = torch.empty_like(y)
        for k in range(K - 1, -1, -1):
            first = k == K - 1
            bufs.fwd(geom, xs[k], add=y, add_scale=-1.0, out=r, config=config)       # r_k (recomputed)
            bufs.fwd(geom, g, out=t, config=config)                                 # t = A g_{k+1}
            dot(t, r, result=dalpha, scale=-1.0, accumulate=not first, workspace=bufs.dws)
            axpby(t, dy32, 1.0, alpha_dev=a, beta=0.0 if first else 1.0)            # dy += alpha t
            bufs.adj(geom, t, op_scale=-1.0, op_scale_dev=a, add=g, add_scale=1.0, out=g,
                     config=config)                                                  # g_k in place
        dy = None
        if ctx.needs_input_grad[0]:
            dy = torch.empty_like(y)
            axpby(dy32, dy, 1.0, beta=0.0)
        return dy, dalpha.reshape(a.shape) if ctx.needs_input_grad[1] else None, \
            g if ctx.needs_input_grad[2] else None, None, None, None


class Landweber:
    """The paper's solver interface: ``Landweber(radon)``, ``estimate_alpha``, ``run``."""

    def __init__(self, radon, config=None):
        self.geometry: Geometry = radon.geometry if hasattr(radon, "geometry") else radon
        self.config = config if config is not None else getattr(radon, "config", None)

    def estimate_alpha(self, img_size: int | None = None, device=None, n_iter: int = 20,
                       v0: torch.Tensor | None = None, seed: int = 0) -> torch.Tensor:
        """The step size alpha = 1 / lambda_max(A^T A) as a one-element float32 device tensor, from
        ``n_iter`` power steps (the paper's call ``estimate_alpha(image_size, device)``, whose result
        is then scaled, e.g. by 0.95).  ``img_size``, if given, must be the geometry's N."""
        if img_size is not None and int(img_size) != self.geometry.n:
            raise ValueError("img_size %d does not match the geometry's %d" % (int(img_size), self.geometry.n))
        alpha, _ = self.power(n_iter, v0=v0, seed=seed, device=device)
        return alpha

    def power(self, iterations: int = 20, v0: torch.Tensor | None = None, seed: int = 0, device=None):
        """(alpha, lambda) from ``iterations`` power steps, as one-element float32 device tensors.

        ``v0`` is the start vector (float32 N x N on the GPU); if omitted it is drawn N(0, 1) from
        ``numpy.random.default_rng(seed)`` on the host and copied over.
        """
        g = self.geometry
        if v0 is None:
            dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
            z = np.random.default_rng(seed).standard_normal((g.n, g.n)).astype(np.float32)
            v0 = torch.from_numpy(z).to(dev)
        lam, alpha = power_iteration(g, v0, iterations)
        return alpha, lam

    def run(self, x0: torch.Tensor, y: torch.Tensor, alpha, iterations: int) -> torch.Tensor:
        """x_K; differentiable w.r.t. ``y``, ``alpha`` (a float32 device tensor) and ``x0``."""
        if x0.dtype != y.dtype:
            raise ValueError("x0 and y must share a dtype")
        a = _alpha_tensor(alpha, y.device)
        return LandweberFunction.apply(y, a, x0, self.geometry, int(iterations), self.config)


def landweber(geom, x0, y, alpha, iterations: int) -> torch.Tensor:
    """Functional form of ``Landweber(geom).run``."""
    return Landweber(geom).run(x0, y, alpha, iterations)
