"""FP64 CPU oracle for the discrete Radon transform (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never touches it and it
never touches the CUDA library: it has its own geometry defaults, its own ray
construction and its own interpolation (``radon_oracle.c``), compiled with gcc
in IEEE double precision.

Readings of the paper that this oracle encodes (each one is also listed with its
justification in the design notes):

* geometry conventions of Sections 3.1.1 / 3.1.2 -- see ``radon_oracle.c``;
* ``det_count`` defaults to the image size, ``det_spacing`` to 1 (Section 3.1.1);
* fan beam: ``det_distance`` defaults to ``source_distance`` and ``det_spacing``
  to the magnified image width over the detector count,
  ``(S + Ddet) / S * N / D`` (Section 3.1.2; reproduces the worked value 2.0);
* Landweber iteration ``x <- x - alpha A^T (A x - y)`` (Section 4.2) with the
  step from a power iteration on ``A^T A`` (Section 4.2), and its reverse mode;
* filtered backprojection (Section 3.1.3): each view's projection is filtered in
  the frequency domain by the DFT of the zero-padded band-limited ramp kernel of
  Kak & Slaney, Chapter 3, Eq. 61, times a window, then backprojected with the
  exact adjoint; the scale pi / V makes ``adjoint(filter_sinogram(A x)) ~ x``;
* CGNE (Section 4.2, after Hanke's "Conjugate gradient type methods for ill-posed
  problems"): conjugate gradients on the normal equation A^T A x = A^T y, which
  minimises |A x - y| over x_0 + K_k(A^T A, A^T r_0); CG for a symmetric positive
  (semi-)definite operator.  Every image of a batch is its own problem;
* the pixel-driven interpolating backprojector (the kind the paper compares with,
  Section 3.1): per view, the sinogram linearly interpolated at the detector
  coordinate of the pixel centre, weighted by the density of rays there
  (|grad t|, detector bins per pixel) so that it approximates the exact adjoint.

Parity status of every function is pinned by tests in ``tests/test_oracle_*.py``
(closed forms, exact symmetries, analytic projections, dense-matrix transposes,
finite differences).
"""

from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "radon_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``radon_oracle.c`` into ``liboracle.so`` (gcc, -O2, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _CGeom(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("n_angles", ctypes.c_int),
        ("angles", ctypes.POINTER(ctypes.c_double)),
        ("det_count", ctypes.c_int),
        ("det_spacing", ctypes.c_double),
        ("step", ctypes.c_double),
        ("fan", ctypes.c_int),
        ("source_distance", ctypes.c_double),
        ("det_distance", ctypes.c_double),
    ]


def _bind(lib):
    P = ctypes.POINTER
    lib.oracle_ray.argtypes = [P(_CGeom), ctypes.c_int, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double)]
    lib.oracle_sample_count.argtypes = [P(_CGeom)]
    lib.oracle_sample_count.restype = ctypes.c_int64
    lib.oracle_ray_sample_counts.argtypes = [P(_CGeom), P(ctypes.c_int64)]
    lib.oracle_forward.argtypes = [P(_CGeom), P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int]
    lib.oracle_adjoint.argtypes = [P(_CGeom), P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int]
    lib.oracle_num_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def using_library(path: str):
    """Test hook: run this wrapper against another build of the oracle source (planted mistakes)."""
    global _lib
    saved = _load()
    _lib = _bind(ctypes.CDLL(os.path.abspath(path)))
    try:
        yield
    finally:
        _lib = saved


@dataclass
class Geometry:
    """Oracle geometry.  ``kind`` is "parallel" or "fan"; ``None`` fields take the paper's defaults."""

    kind: str
    n: int
    angles: np.ndarray
    det_count: int | None = None
    det_spacing: float | None = None
    step: float = 1.0
    source_distance: float = 0.0
    det_distance: float | None = None
    _c: _CGeom = field(default=None, repr=False)
    _angles64: np.ndarray = field(default=None, repr=False)

    def __post_init__(self):
        if self.kind not in ("parallel", "fan"):
            raise ValueError("kind must be 'parallel' or 'fan'")
        self._angles64 = np.ascontiguousarray(np.asarray(self.angles, dtype=np.float64))
        if self.det_count is None or self.det_count <= 0:
            self.det_count = self.n                      # Section 3.1.1: 512 detectors for N = 512
        if self.kind == "fan":
            if self.source_distance <= 0:
                raise ValueError("fan beam needs source_distance > 0")
            if self.det_distance is None or self.det_distance <= 0:
                self.det_distance = self.source_distance  # Section 3.1.2 default
            if self.det_spacing is None or self.det_spacing <= 0:
                # Section 3.1.2: smallest spacing whose bins span the magnified image width
                self.det_spacing = (self.source_distance + self.det_distance) / self.source_distance \
                    * self.n / self.det_count
        else:
            if self.det_spacing is None or self.det_spacing <= 0:
                self.det_spacing = 1.0                   # Section 3.1.1 default
            self.det_distance = 0.0 if self.det_distance is None else self.det_distance
        if self.step is None or self.step <= 0:
            self.step = 1.0
        self._c = _CGeom(int(self.n), int(self._angles64.size),
                         self._angles64.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         int(self.det_count), float(self.det_spacing), float(self.step),
                         1 if self.kind == "fan" else 0, float(self.source_distance),
                         float(self.det_distance or 0.0))

    @property
    def n_angles(self) -> int:
        return int(self._angles64.size)

    @property
    def sino_shape(self) -> tuple[int, int]:
        return (self.n_angles, int(self.det_count))

    @classmethod
    def from_args(cls, args: dict) -> "Geometry":
        a = dict(args)
        kind = a.pop("kind")
        return cls(kind=kind, **a)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def ray(g: Geometry, v: int, d: int) -> tuple[np.ndarray, np.ndarray]:
    """Origin m (closest point to the rotation centre) and unit direction u of ray (v, d)."""
    m = np.zeros(2)
    u = np.zeros(2)
    _load().oracle_ray(ctypes.byref(g._c), v, d, _dp(m), _dp(u))
    return m, u


def sample_count(g: Geometry) -> int:
    """Samples of all rays of one image: the throughput unit."""
    return int(_load().oracle_sample_count(ctypes.byref(g._c)))


def ray_sample_counts(g: Geometry) -> np.ndarray:
    out = np.zeros(g.sino_shape, dtype=np.int64)
    _load().oracle_ray_sample_counts(ctypes.byref(g._c), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return out


def forward(g: Geometry, img: np.ndarray) -> np.ndarray:
    """A x in FP64; ``img`` is [N,N] or [B,N,N]."""
    x = np.ascontiguousarray(np.asarray(img, dtype=np.float64))
    single = x.ndim == 2
    if single:
        x = x[None]
    if x.shape[1:] != (g.n, g.n):
        raise ValueError("image shape %s does not match N=%d" % (x.shape, g.n))
    out = np.zeros((x.shape[0],) + g.sino_shape)
    if x.shape[0]:
        _load().oracle_forward(ctypes.byref(g._c), _dp(x), _dp(out), x.shape[0])
    return out[0] if single else out


def adjoint(g: Geometry, sino: np.ndarray) -> np.ndarray:
    """A^T y in FP64 (literal scatter); ``sino`` is [V,D] or [B,V,D]."""
    y = np.ascontiguousarray(np.asarray(sino, dtype=np.float64))
    single = y.ndim == 2
    if single:
        y = y[None]
    if y.shape[1:] != g.sino_shape:
        raise ValueError("sinogram shape %s does not match %s" % (y.shape, g.sino_shape))
    out = np.zeros((y.shape[0], g.n, g.n))
    if y.shape[0]:
        _load().oracle_adjoint(ctypes.byref(g._c), _dp(y), _dp(out), y.shape[0])
    return out[0] if single else out


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def dense_matrix(g: Geometry) -> np.ndarray:
    """Dense A ([V*D, N*N]) by projecting every unit impulse (small N only)."""
    npix = g.n * g.n
    eye = np.eye(npix).reshape(npix, g.n, g.n)
    cols = forward(g, eye).reshape(npix, -1)
    return cols.T.copy()


def dense_matrix_adjoint(g: Geometry) -> np.ndarray:
    """Dense A^T ([N*N, V*D]) by back-projecting every unit sinogram impulse (small sizes only)."""
    nsino = g.n_angles * g.det_count
    eye = np.eye(nsino).reshape((nsino,) + g.sino_shape)
    cols = adjoint(g, eye).reshape(nsino, -1)
    return cols.T.copy()


# ---------------------------------------------------------------------------
# Landweber iteration (Section 4.2) and its reverse mode.
# ---------------------------------------------------------------------------

def power_iteration(g: Geometry, iterations: int, seed: int) -> float:
    """Rayleigh-quotient estimate of lambda_max(A^T A) after ``iterations`` steps from a seeded N(0,1) start."""
    z = np.random.default_rng(seed).standard_normal((g.n, g.n))
    z /= np.linalg.norm(z)
    lam = 0.0
    for _ in range(iterations):
        w = adjoint(g, forward(g, z))
        lam = float(np.vdot(z, w))   # Rayleigh quotient, |z| = 1
        z = w / np.linalg.norm(w)
    return lam


def landweber(g: Geometry, x0: np.ndarray, y: np.ndarray, alpha: float, iterations: int,
              keep: bool = False):
    """x_{k+1} = x_k - alpha * A^T (A x_k - y); returns x_K (and all iterates if ``keep``)."""
    xs = [np.asarray(x0, dtype=np.float64)]
    for _ in range(iterations):
        x = xs[-1]
        xs.append(x - alpha * adjoint(g, forward(g, x) - y))
    return (xs[-1], xs) if keep else xs[-1]


def landweber_grads(g: Geometry, x0, y, alpha: float, iterations: int, x_true):
    """Loss L = ||x_K - x_true||^2 and its gradients w.r.t. y and alpha (hand-derived reverse mode).

    With r_k = A x_k - y and x_{k+1} = x_k - alpha A^T r_k:
      g_K = dL/dx_K = 2 (x_K - x_true);  g_k = g_{k+1} - alpha A^T A g_{k+1};
      dL/dy     = sum_k alpha * A g_{k+1};
      dL/dalpha = - sum_k <g_{k+1}, A^T r_k>.
    """
    xK, xs = landweber(g, x0, y, alpha, iterations, keep=True)
    loss = float(np.sum((xK - x_true) ** 2))
    gk = 2.0 * (xK - x_true)
    dy = np.zeros_like(np.asarray(y, dtype=np.float64))
    dalpha = 0.0
    for k in range(iterations - 1, -1, -1):
        r = forward(g, xs[k]) - y
        dalpha -= float(np.vdot(gk, adjoint(g, r)))
        Ag = forward(g, gk)
        dy += alpha * Ag
        gk = gk - alpha * adjoint(g, Ag)
    return loss, dy, dalpha


FILTERS = ("ram-lak", "shepp-logan", "cosine", "hamming", "hann")


def ramp_kernel(m: np.ndarray) -> np.ndarray:
    """Band-limited ramp filter at integer offsets m (unit detector spacing), Kak & Slaney Ch. 3
    Eq. 61: 1/4 at m = 0, 0 at even m, -1 / (pi^2 m^2) at odd m."""
    m = np.asarray(m, dtype=np.int64)
    h = np.zeros(m.shape, dtype=np.float64)
    h[m == 0] = 0.25
    odd = (m % 2) != 0
    h[odd] = -1.0 / (np.pi ** 2 * m[odd].astype(np.float64) ** 2)
    return h


def filter_length(det_count: int) -> int:
    """Zero-padded length: the smallest power of two >= 2 D - 1, so that the circular convolution
    of the padded projection equals the linear one."""
    p = 1
    while p < 2 * det_count - 1:
        p *= 2
    return max(p, 2)


def window(name: str, f: np.ndarray) -> np.ndarray:
    """Frequency window at normalised frequency f in [-1/2, 1/2] cycles per detector bin."""
    f = np.asarray(f, dtype=np.float64)
    if name == "ram-lak":
        return np.ones_like(f)
    if name == "shepp-logan":
        return np.sinc(f)                      # sin(pi f) / (pi f)
    if name == "cosine":
        return np.cos(np.pi * f)
    if name == "hamming":
        return 0.54 + 0.46 * np.cos(2 * np.pi * f)
    if name == "hann":
        return 0.5 + 0.5 * np.cos(2 * np.pi * f)
    raise ValueError("unknown filter %r (one of %s)" % (name, ", ".join(FILTERS)))


def frequency_filter(name: str, det_count: int) -> np.ndarray:
    """The length-P Fourier filter: DFT of the zero-padded spatial ramp kernel times the window."""
    p = filter_length(det_count)
    m = np.arange(p)
    m = np.where(m <= p // 2, m, m - p)        # offsets of the circular layout
    ramp = np.fft.fft(ramp_kernel(m)).real     # the kernel is even: the DFT is real
    return ramp * window(name, np.fft.fftfreq(p))


def filter_sinogram(g: Geometry, sino: np.ndarray, name: str = "ram-lak") -> np.ndarray:
    """(pi / V) times each view's projection filtered along the detector: zero-pad to P, FFT,
    multiply by the Fourier filter, inverse FFT, keep the first D bins."""
    y = np.asarray(sino, dtype=np.float64)
    D = y.shape[-1]
    p = filter_length(D)
    H = frequency_filter(name, D)
    Y = np.fft.fft(y, n=p, axis=-1)
    q = np.fft.ifft(Y * H, axis=-1).real[..., :D]
    return (np.pi / g.n_angles) * q


def fbp(g: Geometry, sino: np.ndarray, name: str = "ram-lak") -> np.ndarray:
    """Filtered backprojection: the exact adjoint of the filtered sinogram."""
    return adjoint(g, filter_sinogram(g, sino, name))


def _per_item_dot(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Inner products of the items of a batch (leading axis), FP64."""
    return np.sum(a.reshape(a.shape[0], -1) * b.reshape(b.shape[0], -1), axis=1)


def cgne(g: Geometry, x0: np.ndarray, y: np.ndarray, iterations: int, history: bool = False):
    """CG on A^T A x = A^T y, one problem per image (x0 [B,N,N] or [N,N], y the matching sinograms).

    r = y - A x, s = A^T r, p = s, gamma = |s|^2; per step: q = A p, alpha = gamma / |q|^2,
    x += alpha p, r -= alpha q, s = A^T r, gamma' = |s|^2, p = s + (gamma' / gamma) p.
    Returns x_K (and the list of residual norms |y - A x_k| per item if ``history``)."""
    single = np.ndim(x0) == 2
    x = np.array(x0, dtype=np.float64, copy=True)
    yy = np.asarray(y, dtype=np.float64)
    if single:
        x, yy = x[None], yy[None]
    r = yy - forward(g, x)
    s = adjoint(g, r)
    p = s.copy()
    gamma = _per_item_dot(s, s)
    hist = [np.sqrt(_per_item_dot(r, r))]
    for _ in range(iterations):
        q = forward(g, p)
        qq = _per_item_dot(q, q)
        alpha = np.where(qq > 0, gamma / np.where(qq > 0, qq, 1.0), 0.0)
        x += alpha[:, None, None] * p
        r -= alpha[:, None, None] * q
        s = adjoint(g, r)
        gnew = _per_item_dot(s, s)
        beta = np.where(gamma > 0, gnew / np.where(gamma > 0, gamma, 1.0), 0.0)
        p = s + beta[:, None, None] * p
        gamma = gnew
        hist.append(np.sqrt(_per_item_dot(r, r)))
    out = x[0] if single else x
    return (out, hist) if history else out


def cg(apply_op, x0: np.ndarray, b: np.ndarray, iterations: int):
    """Conjugate gradients for M x = b with M symmetric positive (semi-)definite, given as
    ``apply_op`` on a batch [B, ...]; one problem per item."""
    x = np.array(x0, dtype=np.float64, copy=True)
    r = np.asarray(b, dtype=np.float64) - apply_op(x)
    p = r.copy()
    rr = _per_item_dot(r, r)
    expand = (slice(None),) + (None,) * (x.ndim - 1)
    for _ in range(iterations):
        mp = apply_op(p)
        pmp = _per_item_dot(p, mp)
        alpha = np.where(pmp > 0, rr / np.where(pmp > 0, pmp, 1.0), 0.0)
        x += alpha[expand] * p
        r -= alpha[expand] * mp
        rnew = _per_item_dot(r, r)
        beta = np.where(rr > 0, rnew / np.where(rr > 0, rr, 1.0), 0.0)
        p = r + beta[expand] * p
        rr = rnew
    return x


def detector_coordinate(g: Geometry, v: int):
    """Continuous detector index t(x, y) of every pixel centre for view v, and |grad t| (bins per
    pixel): parallel t = (c . n) / ds + (D - 1) / 2; fan (source -S u, flat detector at Ddet along
    u): s = (S + Ddet) (c . n) / (c . u + S), the intersection of the source-pixel line with the
    detector, t = s / ds + (D - 1) / 2."""
    th = float(g.angles[v])
    n = np.array([np.cos(th), np.sin(th)])
    u = np.array([-np.sin(th), np.cos(th)])
    c0 = (g.n - 1) / 2.0
    X, Y = np.meshgrid(np.arange(g.n) - c0, np.arange(g.n) - c0)     # [i, j] -> (x = j - c0, y = i - c0)
    cn = X * n[0] + Y * n[1]
    ds = g.det_spacing
    if g.kind == "fan":
        S, Dd = g.source_distance, g.det_distance
        cu = X * u[0] + Y * u[1]
        den = cu + S
        s = (S + Dd) * cn / den
        grad = (S + Dd) * np.sqrt(den ** 2 + cn ** 2) / den ** 2
    else:
        s = cn
        grad = np.ones_like(cn)
    return s / ds + (g.det_count - 1) / 2.0, grad / ds


def backproject_interpolating(g: Geometry, sino: np.ndarray) -> np.ndarray:
    """sum_v |grad t_v| * (sino[v] linearly interpolated at t_v(pixel)), bins outside [0, D) zero."""
    y = np.asarray(sino, dtype=np.float64)
    single = y.ndim == 2
    if single:
        y = y[None]
    out = np.zeros((y.shape[0], g.n, g.n))
    D = g.det_count
    for v in range(g.n_angles):
        t, w = detector_coordinate(g, v)
        i0 = np.floor(t).astype(np.int64)
        f = t - i0
        row = np.concatenate([y[:, v, :], np.zeros((y.shape[0], 1))], axis=1)   # index D reads as zero
        lo = np.where((i0 >= 0) & (i0 < D), i0, D)
        hi = np.where((i0 + 1 >= 0) & (i0 + 1 < D), i0 + 1, D)
        out += w * ((1.0 - f) * row[:, lo] + f * row[:, hi])
    return out[0] if single else out


__all__ = [
    "Geometry", "build", "ray", "sample_count", "ray_sample_counts", "forward", "adjoint",
    "num_threads", "dense_matrix", "dense_matrix_adjoint", "power_iteration", "landweber",
    "landweber_grads", "FILTERS", "ramp_kernel", "filter_length", "window", "frequency_filter",
    "filter_sinogram", "fbp", "cgne", "cg", "detector_coordinate", "backproject_interpolating",
]

