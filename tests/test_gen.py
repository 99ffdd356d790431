"""Pins of the input generator's cubic B-spline bases (the marginal designs of Sec. 4.1)."""
import os

import numpy as np
import pytest

import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_textbook_values():
    tab = np.loadtxt(os.path.join(GOLDEN, "cubic_bspline_uniform.txt"))
    B = gen.cubic_bspline_basis(3, 4)
    np.testing.assert_allclose(B, tab[:, 1:], rtol=0, atol=1e-15)


@pytest.mark.parametrize("n,p", [(20, 8), (128, 20), (600, 60), (96, 30), (7, 5), (365, 40)])
def test_partition_of_unity_and_support(n, p):
    B = gen.cubic_bspline_basis(n, p)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-13)
    assert np.all(B >= -1e-15)
    assert np.all((np.abs(B) > 1e-15).sum(axis=1) <= 4)


@pytest.mark.parametrize("n,p", [(20, 8), (37, 11), (128, 20)])
def test_matches_scipy_bspline(n, p):
    interp = pytest.importorskip("scipy.interpolate")
    h = 1.0 / (p - 3)
    t = np.arange(-3, p + 1) * h
    x = np.linspace(0, 1, n)
    ref = np.zeros((n, p))
    for j in range(p):
        c = np.zeros(p)
        c[j] = 1.0
        ref[:, j] = interp.BSpline(t, c, 3, extrapolate=False)(x)
    ref = np.nan_to_num(ref)
    np.testing.assert_allclose(gen.cubic_bspline_basis(n, p), ref, atol=1e-13)


def test_workloads_are_seeded_and_shaped():
    a = gen.make_workload(0)
    b = gen.make_workload(0)
    np.testing.assert_array_equal(a.Y, b.Y)
    assert a.Y.shape == (20, 20, 20) and a.p == (8, 8, 8)
    assert np.count_nonzero(a.theta_true) == round(0.1 * 512)
    c = gen.make_workload(2, n=(24, 20, 30), p=(6, 6, 8))
    assert c.Y.shape == (30, 20, 24)
    assert int((c.W == 0).sum()) == round(0.1 * c.Y.size)
    assert c.eta_true.min() >= -2 - 1e-12 and c.eta_true.max() <= 4 + 1e-12
