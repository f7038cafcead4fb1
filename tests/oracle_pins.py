"""Pins for the FP64 oracle: checks against facts that do not come from the oracle itself.

Each ``pin_*`` function returns the worst relative error it saw; ``check_all``
runs every pin against its tolerance.  The same functions run against the real
oracle (``test_oracle_pins.py``) and against copies of the oracle with planted
mistakes (``test_oracle_mutants.py``), which must each fail at least one pin.

What pins what:
  * theta = 0 / pi/2 closed forms (column / row sums, linear interpolation across
    detectors): pixel-centre convention, detector direction and spacing, the
    step factor h, the support box, which axis is which.
  * theta = pi/4 with ds = h = 1/sqrt(2): samples land on the half-integer grid;
    the value is an integer-index sum over the 2x-upsampled image.
  * exact symmetries (opposite view, 90-degree rotation, transpose; fan analogues).
  * analytic line integrals of a Gaussian (parallel and fan) and of ellipses:
    angle direction, source / detector placement, scaling.
  * mass conservation, the sample-count closed form, the paper's worked fan-beam
    default spacing (golden fixture), the fan -> parallel limit.
  * dense A from impulses vs dense A^T from impulses, and the dot-product test:
    the adjoint is the transpose of the forward.
  * power iteration vs numpy.linalg.eigvalsh; Landweber reverse mode vs finite
    differences.
"""

from __future__ import annotations

import json
import math
import os

import numpy as np

import oracle as O
from synth import gaussian_blob, random_ellipses, rasterize_ellipses, uniform_angles

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _worse(worst, val):
    """The larger of two errors; NaN wins (a broken oracle must not pass as a zero error)."""
    val = float(val)
    return val if not val <= worst else worst


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = max(np.linalg.norm(b), 1e-300)
    return float(np.linalg.norm(a - b) / den)


def _rand_img(n, seed):
    return np.random.default_rng(seed).uniform(0.0, 1.0, (n, n))


def _lerp_zero_outside(values, f):
    """Linear interpolation of ``values`` (index 0..len-1, zero outside) at fractional indices ``f``."""
    idx = np.arange(-1, len(values) + 1, dtype=np.float64)
    vals = np.concatenate([[0.0], values, [0.0]])
    return np.interp(f, idx, vals, left=0.0, right=0.0)


# --------------------------------------------------------------------------- closed forms

def pin_theta0(n=64, d=91, ds=1.0, h=1.0, seed=1):
    """theta = 0: y(d) = linear interpolation of the column sums at x = s_d (h = 1/m)."""
    x = _rand_img(n, seed)
    g = O.Geometry("parallel", n, np.array([0.0]), d, ds, h)
    y = O.forward(g, x)[0]
    s = (np.arange(d) - (d - 1) / 2.0) * ds
    expect = _lerp_zero_outside(x.sum(axis=0), s + (n - 1) / 2.0)
    return _rel(y, expect)


def pin_theta_half_pi(n=48, d=60, ds=0.8, h=0.5, seed=2):
    """theta = pi/2: rays run along -x at y = s_d; y(d) = interpolated row sums."""
    x = _rand_img(n, seed)
    g = O.Geometry("parallel", n, np.array([math.pi / 2]), d, ds, h)
    y = O.forward(g, x)[0]
    s = (np.arange(d) - (d - 1) / 2.0) * ds
    expect = _lerp_zero_outside(x.sum(axis=1), s + (n - 1) / 2.0)
    return _rel(y, expect)


def pin_theta_quarter_pi(n=31, d=61, seed=3):
    """theta = pi/4, ds = h = 1/sqrt 2: sample (d', k) sits at ((d'-k)/2, (d'+k)/2) + c0.

    Even d'-k: an integer grid point, the value is one pixel.  Odd: a cell centre,
    the value is the mean of four pixels.  Pure integer indexing, no interpolation code.
    """
    assert n % 2 == 1 and d % 2 == 1
    x = _rand_img(n, seed)
    h = math.sqrt(0.5)
    g = O.Geometry("parallel", n, np.array([math.pi / 4]), d, h, h)
    y = O.forward(g, x)[0]
    xp = np.zeros((n + 2, n + 2))
    xp[1:-1, 1:-1] = x                      # xp[i+1, j+1] = x[i, j]; zero border
    c2 = n - 1                              # 2 * (N-1)/2
    expect = np.zeros(d)
    for di in range(d):
        dp = di - (d - 1) // 2
        tot = 0.0
        for k in range(-4 * n, 4 * n + 1):
            X2 = dp - k + c2                # 2 * fx
            Y2 = dp + k + c2                # 2 * fy
            if not (-2 < X2 < 2 * n and -2 < Y2 < 2 * n):
                continue                    # outside the open support box
            if X2 % 2 == 0:
                tot += xp[Y2 // 2 + 1, X2 // 2 + 1]
            else:
                i0, j0 = (Y2 - 1) // 2, (X2 - 1) // 2
                tot += 0.25 * (xp[i0 + 1, j0 + 1] + xp[i0 + 1, j0 + 2] + xp[i0 + 2, j0 + 1] + xp[i0 + 2, j0 + 2])
        expect[di] = h * tot
    return _rel(y, expect)


def pin_sample_count_theta0(n=20, d=26, ds=0.9, h=0.5):
    """theta = 0: S = #{d : |s_d| < (N+1)/2} * #{k : |k h| < (N+1)/2}."""
    g = O.Geometry("parallel", n, np.array([0.0]), d, ds, h)
    half = (n + 1) / 2.0
    s = (np.arange(d) - (d - 1) / 2.0) * ds
    nd = int(np.sum(np.abs(s) < half))
    ks = np.arange(-4 * n, 4 * n + 1)
    nk = int(np.sum(np.abs(ks * h) < half))
    return float(abs(O.sample_count(g) - nd * nk))


def pin_mass_theta0(n=40, d=50):
    """theta = 0, ds = h = 1, detectors covering the support: h ds sum_d y = sum x exactly."""
    x = _rand_img(n, 4)
    g = O.Geometry("parallel", n, np.array([0.0]), d, 1.0, 1.0)
    y = O.forward(g, x)[0]
    return abs(y.sum() - x.sum()) / x.sum()


def pin_mass_all_angles(n=40, d=64, views=16):
    """Any angle: the detector sum approximates the image mass (aliasing of the tent, < 1e-2)."""
    x = rasterize_ellipses(random_ellipses(n, 4, 5), n, 2)
    g = O.Geometry("parallel", n, uniform_angles(views, math.pi), d, 1.0, 1.0)
    y = O.forward(g, x)
    return float(np.max(np.abs(y.sum(axis=1) - x.sum())) / x.sum())


# --------------------------------------------------------------------------- symmetries

def pin_symmetry_parallel(n=24, d=37, seed=6):
    x = _rand_img(n, seed)
    th = np.array([0.17, 0.9, 1.3, 2.2])
    errs = []
    g = O.Geometry("parallel", n, np.concatenate([th, th + math.pi, th + math.pi / 2, math.pi / 2 - th]), d, 1.0, 1.0)
    y = O.forward(g, x)
    yT = O.forward(g, x.T.copy())
    yR = O.forward(g, np.rot90(x).copy())
    m = len(th)
    errs.append(_rel(y[m:2 * m], y[:m, ::-1]))           # y(t + pi, d) = y(t, D-1-d)
    errs.append(_rel(yR[:m], y[2 * m:3 * m]))             # rot90(x) at t = x at t + pi/2
    errs.append(_rel(yT[:m], y[3 * m:4 * m]))             # transpose at t = x at pi/2 - t
    return max(errs)


def pin_symmetry_fan(n=24, d=41, seed=7):
    x = _rand_img(n, seed)
    th = np.array([0.2, 1.1, 2.5, 4.0])
    g = O.Geometry("fan", n, np.concatenate([th, th + math.pi / 2, 1.5 * math.pi - th]), d, 0.9, 1.0,
                   source_distance=40.0, det_distance=25.0)
    y = O.forward(g, x)
    yT = O.forward(g, x.T.copy())
    yR = O.forward(g, np.rot90(x).copy())
    m = len(th)
    return max(_rel(yR[:m], y[m:2 * m]),                  # rigid rotation of the whole set-up
               _rel(yT[:m], y[2 * m:3 * m, ::-1]))        # mirror: source to 3pi/2 - t, bins reversed


# --------------------------------------------------------------------------- analytic projections

def _gauss_line_integral(amp, sigma, dist):
    return amp * sigma * math.sqrt(2 * math.pi) * np.exp(-dist ** 2 / (2 * sigma ** 2))


def _gauss_expected(amp, sigma, dist):
    """Line integral L of the Gaussian plus the mean bias of bilinear interpolation.

    Linear interpolation at fraction a overestimates f by a(1-a)/2 f''; over
    uniformly distributed phases that averages to f''/12 per axis, and the line
    integral of the Laplacian is the second derivative of L across the ray:
    E[y] = L + L''/12 with L'' = L (dist^2/sigma^4 - 1/sigma^2).
    """
    L = _gauss_line_integral(amp, sigma, dist)
    return L + L * (dist ** 2 / sigma ** 4 - 1.0 / sigma ** 2) / 12.0


def pin_gaussian_parallel(n=96, d=140, views=24, sigma=6.0, c=(9.0, -13.0)):
    """Discrete projection of a sampled Gaussian vs its exact line integral along x.n = s_d."""
    x = gaussian_blob(n, c[0], c[1], sigma)
    th = uniform_angles(views, math.pi) + 0.013
    g = O.Geometry("parallel", n, th, d, 0.75, 1.0)
    y = O.forward(g, x)
    s = (np.arange(d) - (d - 1) / 2.0) * 0.75
    dist = (c[0] * np.cos(th) + c[1] * np.sin(th))[:, None] - s[None, :]
    return _rel(y, _gauss_expected(1.0, sigma, dist))


def pin_gaussian_fan(n=96, d=120, views=24, sigma=6.0, c=(-11.0, 7.0), src=300.0, det=200.0, ds=1.3):
    """Fan beam: exact Gaussian line integral along the line from -S u to Ddet u + s_d n."""
    x = gaussian_blob(n, c[0], c[1], sigma)
    th = uniform_angles(views, 2 * math.pi) + 0.021
    g = O.Geometry("fan", n, th, d, ds, 1.0, source_distance=src, det_distance=det)
    y = O.forward(g, x)
    s = (np.arange(d) - (d - 1) / 2.0) * ds
    ux, uy = -np.sin(th)[:, None], np.cos(th)[:, None]
    nx, ny = np.cos(th)[:, None], np.sin(th)[:, None]
    ax, ay = -src * ux, -src * uy                          # source
    bx, by = det * ux + s * nx, det * uy + s * ny          # bin centre
    ex, ey = bx - ax, by - ay
    dist = np.abs(ex * (c[1] - ay) - ey * (c[0] - ax)) / np.hypot(ex, ey)
    return _rel(y, _gauss_expected(1.0, sigma, dist))


def pin_ellipse_parallel(n=96, d=136, views=20):
    """Supersampled ellipses vs the analytic ellipse projection (pixelisation error ~ 1e-2)."""
    ells = random_ellipses(n, 3, 8)
    x = rasterize_ellipses(ells, n, 4)
    th = uniform_angles(views, math.pi) + 0.05
    g = O.Geometry("parallel", n, th, d, 1.0, 1.0)
    y = O.forward(g, x)
    s = (np.arange(d) - (d - 1) / 2.0)[None, :]
    expect = np.zeros_like(y)
    for e in ells:
        sp = s - (e.x0 * np.cos(th) + e.y0 * np.sin(th))[:, None]
        a2 = (e.a ** 2 * np.cos(th - e.phi) ** 2 + e.b ** 2 * np.sin(th - e.phi) ** 2)[:, None]
        inside = sp ** 2 < a2
        expect += np.where(inside, 2 * e.rho * e.a * e.b * np.sqrt(np.where(inside, a2 - sp ** 2, 0.0)) / a2, 0.0)
    return _rel(y, expect)


def pin_fan_default_spacing():
    """Golden: the paper's worked fan-beam example gives det_spacing 2.0 (Section 3.1.2)."""
    with open(os.path.join(GOLDEN, "fan_default_spacing.json")) as f:
        gold = json.load(f)
    g = O.Geometry("fan", gold["n"], uniform_angles(4, 2 * math.pi), gold["det_count"], None, 1.0,
                   source_distance=gold["source_distance"])
    return abs(g.det_spacing - gold["det_spacing"]) + abs(g.det_distance - gold["det_distance"])


def pin_fan_central_ray(n=40, d=51):
    """The central fan ray (s = 0) is the parallel ray through the centre: identical samples."""
    x = _rand_img(n, 9)
    th = np.array([0.3, 1.7, 3.9])
    gf = O.Geometry("fan", n, th, d, 1.0, 1.0, source_distance=70.0, det_distance=30.0)
    gp = O.Geometry("parallel", n, th, d, 1.0, 1.0)
    c = (d - 1) // 2
    return _rel(O.forward(gf, x)[:, c], O.forward(gp, x)[:, c])


def pin_fan_parallel_limit(n=40, d=57):
    """Source at 1e10 px and detector through the centre: fan -> parallel."""
    x = rasterize_ellipses(random_ellipses(n, 4, 10), n, 2)
    th = uniform_angles(7, 2 * math.pi) + 0.1
    gf = O.Geometry("fan", n, th, d, 1.0, 1.0, source_distance=1e10, det_distance=1e-6)
    gp = O.Geometry("parallel", n, th, d, 1.0, 1.0)
    return _rel(O.forward(gf, x), O.forward(gp, x))


# --------------------------------------------------------------------------- adjoint

def _small_geoms():
    return [
        O.Geometry("parallel", 8, uniform_angles(6, math.pi) + 0.05, 11, 1.0, 1.0),
        O.Geometry("parallel", 7, uniform_angles(5, math.pi), 9, 0.7, 0.6),
        O.Geometry("fan", 8, uniform_angles(6, 2 * math.pi) + 0.1, 13, 1.1, 1.0,
                   source_distance=20.0, det_distance=12.0),
    ]


def pin_dense_transpose():
    """A from forward impulses equals (A^T from adjoint impulses)^T."""
    worst = 0.0
    for g in _small_geoms():
        A = O.dense_matrix(g)
        At = O.dense_matrix_adjoint(g)
        scale = float(np.max(np.abs(A)))
        if not scale > 0.0:
            return math.inf   # an empty (or non-finite) system matrix fails the pin
        worst = _worse(worst, float(np.max(np.abs(A - At.T))) / scale)
    return worst


def pin_dot_product():
    worst = 0.0
    geoms = _small_geoms() + [O.Geometry("fan", 33, uniform_angles(17, 2 * math.pi), 50, None, 1.0,
                                         source_distance=60.0)]
    for i, g in enumerate(geoms):
        rng = np.random.default_rng(100 + i)
        x = rng.standard_normal((2, g.n, g.n))
        y = rng.standard_normal((2,) + g.sino_shape)
        a = float(np.vdot(O.forward(g, x), y))
        b = float(np.vdot(x, O.adjoint(g, y)))
        worst = _worse(worst, abs(a - b) / max(abs(a), abs(b)))
    return worst


# --------------------------------------------------------------------------- solvers

def pin_power_iteration():
    g = O.Geometry("parallel", 8, uniform_angles(6, math.pi) + 0.05, 11, 1.0, 1.0)
    A = O.dense_matrix(g)
    lam = float(np.linalg.eigvalsh(A.T @ A)[-1])
    est = O.power_iteration(g, 400, seed=3)
    est20 = O.power_iteration(g, 20, seed=3)
    if est20 > lam * (1 + 1e-12):
        return 1.0                               # a Rayleigh quotient never exceeds lambda_max
    return abs(est - lam) / lam


def pin_landweber_fd():
    g = O.Geometry("parallel", 8, uniform_angles(5, math.pi) + 0.05, 11, 1.0, 1.0)
    rng = np.random.default_rng(11)
    xt = rng.uniform(0, 1, (8, 8))
    y = O.forward(g, xt) + 0.01 * rng.standard_normal(g.sino_shape)
    A = O.dense_matrix(g)
    alpha = 0.7 / float(np.linalg.eigvalsh(A.T @ A)[-1])
    K = 3
    x0 = np.zeros((8, 8))
    loss, dy, dalpha = O.landweber_grads(g, x0, y, alpha, K, xt)

    def L(yy, aa):
        return float(np.sum((O.landweber(g, x0, yy, aa, K) - xt) ** 2))

    eps = 1e-6
    dirn = rng.standard_normal(g.sino_shape)
    fd_y = (L(y + eps * dirn, alpha) - L(y - eps * dirn, alpha)) / (2 * eps)
    ea = alpha * 1e-6
    fd_a = (L(y, alpha + ea) - L(y, alpha - ea)) / (2 * ea)
    return max(abs(fd_y - float(np.vdot(dy, dirn))) / abs(fd_y), abs(fd_a - dalpha) / abs(fd_a),
               abs(L(y, alpha) - loss) / loss)


# --------------------------------------------------------------------------- registry

PINS = {
    # name: (function, tolerance)
    "theta0_d91": (lambda: pin_theta0(64, 91, 1.0, 1.0), 1e-13),
    "theta0_d64": (lambda: pin_theta0(64, 64, 1.0, 1.0), 1e-13),
    "theta0_odd_ds07_h05": (lambda: pin_theta0(33, 40, 0.7, 0.5), 1e-13),
    "theta0_ds13_h025": (lambda: pin_theta0(16, 20, 1.3, 0.25), 1e-13),
    "theta_half_pi": (pin_theta_half_pi, 1e-12),
    "theta_quarter_pi": (pin_theta_quarter_pi, 1e-12),
    "sample_count_theta0": (pin_sample_count_theta0, 0.5),
    "sample_count_theta0_boundary": (lambda: pin_sample_count_theta0(20, 22, 1.0, 1.0), 0.5),
    "mass_theta0": (pin_mass_theta0, 1e-13),
    "mass_all_angles": (pin_mass_all_angles, 1e-2),
    "symmetry_parallel": (pin_symmetry_parallel, 1e-12),
    "symmetry_fan": (pin_symmetry_fan, 1e-12),
    "gaussian_parallel": (pin_gaussian_parallel, 8e-4),
    "gaussian_fan": (pin_gaussian_fan, 8e-4),
    "ellipse_parallel": (pin_ellipse_parallel, 3e-2),
    "fan_default_spacing": (pin_fan_default_spacing, 1e-12),
    "fan_central_ray": (pin_fan_central_ray, 1e-12),
    "fan_parallel_limit": (pin_fan_parallel_limit, 1e-4),
    "dense_transpose": (pin_dense_transpose, 1e-13),
    "dot_product": (pin_dot_product, 1e-12),
    "power_iteration": (pin_power_iteration, 1e-8),
    "landweber_fd": (pin_landweber_fd, 1e-6),
}


def run_all(names=None):
    """{name: (value, tolerance, passed)}; a pin that raises counts as failed."""
    out = {}
    for name, (fn, tol) in PINS.items():
        if names is not None and name not in names:
            continue
        try:
            val = float(fn())
            ok = bool(np.isfinite(val) and val <= tol)
        except Exception as exc:  # a broken oracle may fail loudly; that is a caught mistake
            val, ok = repr(exc), False
        out[name] = (val, tol, ok)
    return out
