"""Pins of the oracle's CGNE and CG (Section 4.2; Hanke's conjugate gradient type methods) against
what linear algebra fixes: the k-th CGNE iterate is the least-squares minimiser over the k-th Krylov
space, the k-th CG iterate is the Galerkin solution there and, after n steps, the solution."""

from __future__ import annotations

import math

import numpy as np

import oracle as O
from synth import uniform_angles


def _small():
    g = O.Geometry("parallel", 8, uniform_angles(6, math.pi) + 0.1, 11)
    A = O.dense_matrix(g)                     # [V*D, N*N]
    return g, A


def _krylov(Mop, v, k):
    """Orthonormal basis of span{v, M v, ..., M^(k-1) v} (re-orthogonalised)."""
    basis = []
    w = v.copy()
    for _ in range(k):
        for b in basis:
            w = w - np.dot(b, w) * b
        w = w / np.linalg.norm(w)
        basis.append(w)
        w = Mop(w)
    return np.stack(basis, axis=1)


def test_cgne_iterates_are_krylov_least_squares_minimisers():
    g, A = _small()
    rng = np.random.default_rng(2)
    x0 = rng.normal(size=(g.n, g.n))
    y = rng.normal(size=g.sino_shape)
    r0 = y.ravel() - A @ x0.ravel()
    for k in range(1, 6):
        Vk = _krylov(lambda v: A.T @ (A @ v), A.T @ r0, k)
        c, *_ = np.linalg.lstsq(A @ Vk, r0, rcond=None)
        ref = x0.ravel() + Vk @ c
        got = O.cgne(g, x0, y, k).ravel()
        assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref), k


def test_cgne_residuals_never_increase_and_items_are_independent():
    g, _ = _small()
    rng = np.random.default_rng(5)
    x0 = np.zeros((2, g.n, g.n))
    y = rng.normal(size=(2,) + g.sino_shape)
    x, hist = O.cgne(g, x0, y, 12, history=True)
    h = np.stack(hist)                           # [iters + 1, batch]
    assert np.all(np.diff(h, axis=0) <= 1e-12 * h[0])
    for b in range(2):
        assert np.allclose(O.cgne(g, x0[b], y[b], 12), x[b], rtol=0, atol=1e-12 * np.abs(x[b]).max())


def test_cg_iterates_are_galerkin_solutions_and_converge():
    rng = np.random.default_rng(7)
    n = 12
    Q = np.linalg.qr(rng.normal(size=(n, n)))[0]
    M = Q @ np.diag(np.linspace(1.0, 20.0, n)) @ Q.T
    b = rng.normal(size=(1, n))
    x0 = rng.normal(size=(1, n))
    op = lambda v: v @ M.T                      # noqa: E731  (batch of row vectors)
    r0 = (b - op(x0))[0]
    for k in range(1, 6):
        Vk = _krylov(lambda v: M @ v, r0, k)
        c = np.linalg.solve(Vk.T @ M @ Vk, Vk.T @ r0)
        ref = x0[0] + Vk @ c
        assert np.linalg.norm(O.cg(op, x0, b, k)[0] - ref) <= 1e-9 * np.linalg.norm(ref), k
    assert np.allclose(O.cg(op, x0, b, n)[0], np.linalg.solve(M, b[0]), rtol=1e-8, atol=1e-10)
