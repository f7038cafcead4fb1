"""Plant plausible mistakes in a copy of the oracle's C source; every one must fail a pin.

This shows the pins have teeth: a dropped term, a wrong sign, a transposed operand
or a misplaced geometry element anywhere in the oracle is caught by at least one
of them.  The mutants are built from a copy in a temporary directory; the real
oracle is never modified.
"""

import os
import subprocess

import pytest

import oracle
import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "radon_oracle.c")

# (name, original text, replacement) -- each original must occur exactly once
MUTANTS = [
    ("detector_direction_flipped", "m[0] = s * nx;\n        m[1] = s * ny;", "m[0] = -s * nx;\n        m[1] = -s * ny;"),
    ("detector_centre_off_by_one", "((double)d - 0.5 * (double)(g->det_count - 1))", "((double)d - 0.5 * (double)(g->det_count))"),
    ("pixel_centre_half_shift", "double fx = p[0] + 0.5 * (double)(n - 1);\n    double fy = p[1] + 0.5 * (double)(n - 1);\n    double j0 = floor(fx), i0 = floor(fy);\n    double a = fx - j0, b = fy - i0;\n    long j = (long)j0, i = (long)i0;\n    double v = 0.0;",
     "double fx = p[0] + 0.5 * (double)(n);\n    double fy = p[1] + 0.5 * (double)(n - 1);\n    double j0 = floor(fx), i0 = floor(fy);\n    double a = fx - j0, b = fy - i0;\n    long j = (long)j0, i = (long)i0;\n    double v = 0.0;"),
    ("bilinear_weights_transposed", "double w = (dj ? a : 1.0 - a) * (di ? b : 1.0 - b);\n            v += w", "double w = (dj ? b : 1.0 - b) * (di ? a : 1.0 - a);\n            v += w"),
    ("bilinear_term_dropped", "if (ii < 0 || ii >= n || jj < 0 || jj >= n) continue;\n            double w = (dj ? a : 1.0 - a) * (di ? b : 1.0 - b);\n            v += w",
     "if (ii < 0 || ii >= n || jj < 0 || jj >= n || (di && dj)) continue;\n            double w = (dj ? a : 1.0 - a) * (di ? b : 1.0 - b);\n            v += w"),
    ("step_factor_dropped", "= g->step * acc;", "= acc;"),
    ("box_closed", "return fabs(p[0]) < half && fabs(p[1]) < half;", "return fabs(p[0]) <= half && fabs(p[1]) <= half;"),
    ("box_too_small", "double half = 0.5 * (double)(g->n + 1);", "double half = 0.5 * (double)(g->n);"),
    ("ray_direction_wrong", "double ux = -sin(th), uy = cos(th);", "double ux = sin(th), uy = cos(th);"),
    ("angle_sign_flipped", "double nx = cos(th), ny = sin(th);\n    double ux = -sin(th), uy = cos(th);", "double nx = cos(th), ny = -sin(th);\n    double ux = sin(th), uy = cos(th);"),
    ("fan_source_wrong_side", "double cx = -g->source_distance * ux, cy = -g->source_distance * uy;", "double cx = g->source_distance * ux, cy = g->source_distance * uy;"),
    ("fan_detector_distance_ignored", "double qx = g->det_distance * ux + s * nx, qy = g->det_distance * uy + s * ny;", "double qx = s * nx, qy = s * ny;"),
    ("fan_origin_not_foot", "m[0] = cx - cr * rx;\n    m[1] = cy - cr * ry;", "m[0] = cx;\n    m[1] = cy;"),
    ("adjoint_weights_swapped", "double w = (dj ? a : 1.0 - a) * (di ? b : 1.0 - b);\n            img[ii * n + jj] += w * val;", "double w = (dj ? 1.0 - a : a) * (di ? b : 1.0 - b);\n            img[ii * n + jj] += w * val;"),
    ("adjoint_step_dropped", "double val = g->step * sino[", "double val = sino["),
]


@pytest.mark.parametrize("name,orig,repl", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, orig, repl, tmp_path):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation anchor for {name} not found exactly once"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(orig, repl))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", str(mutated), "-o", str(lib), "-lm"], check=True)
    with oracle.using_library(str(lib)):
        results = P.run_all()
    failed = [k for k, (_, _, ok) in results.items() if not ok]
    assert failed, f"planted mistake '{name}' passed every pin"
