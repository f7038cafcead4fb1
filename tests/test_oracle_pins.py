"""The FP64 oracle against facts that do not come from it (closed forms, symmetries,
analytic projections, dense transposes, library eigenvalues, finite differences)."""

import pytest

import oracle_pins as P


@pytest.mark.parametrize("name", sorted(P.PINS))
def test_pin(name):
    val, tol, ok = P.run_all([name])[name]
    assert ok, f"{name}: {val} > {tol}"
