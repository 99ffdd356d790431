"""Pins of the oracle's SCAD fit by the multistep adaptive lasso (the package's penalty "scad",
Sec. 6.4; the local linear approximation of the SCAD penalty).

* the SCAD derivative has the published piecewise form (lambda up to lambda, linear decay to 0 at
  a lambda, zero beyond), checked pointwise;
* one step is the weighted lasso itself;
* on an orthonormal design the steps converge to the closed-form SCAD thresholding rule of Fan
  and Li (soft threshold up to 2 lambda, the linear middle piece up to a lambda, no shrinkage
  beyond), coordinate by coordinate;
* a planted mistake (the derivative without its (a - 1) denominator) is caught by that rule.
"""
import numpy as np

import gen
import oracle as O


def test_scad_derivative_pieces():
    lam, a = 0.5, 3.7
    t = np.array([0.0, 0.2, 0.5, 0.6, 1.0, 1.85, 2.0, 5.0])
    expect = [0.5, 0.5, 0.5, (1.85 - 0.6) / 2.7, (1.85 - 1.0) / 2.7, 0.0, 0.0, 0.0]
    np.testing.assert_allclose(O.scad_derivative(t, lam, a), expect, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(O.scad_derivative(-t, lam, a), expect, rtol=1e-14, atol=1e-15)


def test_one_step_is_the_lasso():
    pr = gen.random_problem(61, (8, 7, 6), (3, 3, 3), gen.POISSON, basis="normal", pen_w="rand")
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    lmax = O.lambda_max(d)
    lam = 0.2 * lmax
    a, _ = O.gdpg(d, lam, np.zeros(d.pshape), lmax, tol=1e-11)
    b, _, w = O.msa_scad(d, lam, np.zeros(d.pshape), lmax, steps=1, tol=1e-11)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(w, d.pen_w)


def _fan_li(z, lam, a):
    az = np.abs(z)
    soft = np.sign(z) * np.maximum(az - lam, 0.0)
    mid = ((a - 1.0) * z - np.sign(z) * a * lam) / (a - 2.0)
    return np.where(az <= 2 * lam, soft, np.where(az <= a * lam, mid, z))


def _orthonormal(seed):
    rng = np.random.default_rng(seed)
    n, p = (6, 5, 4), (3, 3, 2)
    # X_j = sqrt(n_j) Q_j: X^T X = n I, so f = (1/2n)||y - X theta||^2 is, coordinate by
    # coordinate, (1/2)(theta - z)^2 + const with z = X^T y / n
    Xs = [np.sqrt(n[j]) * np.linalg.qr(rng.standard_normal((n[j], p[j])))[0] for j in range(3)]
    Y = rng.standard_normal(n)
    d = O.GlamData(O.GAUSSIAN, Xs, Y, np.ones(n), np.ones(p))
    z = O.G(Xs, Y) / Y.size
    return d, z


def test_orthonormal_design_reaches_the_scad_rule():
    d, z = _orthonormal(62)
    lam = 0.25 * float(np.max(np.abs(z)))
    lmax = O.lambda_max(d)
    th, _, _ = O.msa_scad(d, lam, np.zeros(d.pshape), lmax, steps=60, tol=1e-12)
    ref = _fan_li(z, lam, O.SCAD_A)
    regions = np.abs(z) / lam
    assert np.any(regions <= 2) and np.any((regions > 2) & (regions <= O.SCAD_A)) and np.any(regions > O.SCAD_A)
    np.testing.assert_allclose(th, ref, atol=1e-9)


def test_planted_missing_denominator_is_caught(monkeypatch):
    d, z = _orthonormal(62)
    lam = 0.25 * float(np.max(np.abs(z)))
    lmax = O.lambda_max(d)
    good = O.glam_oracle.scad_derivative
    monkeypatch.setattr(O.glam_oracle, "scad_derivative",
                        lambda t, l, a=O.SCAD_A: good(t, l, a) * np.where(np.abs(t) <= l, 1.0, a - 1.0))
    th, _, _ = O.glam_oracle.msa_scad(d, lam, np.zeros(d.pshape), lmax, steps=60, tol=1e-12)
    assert not np.allclose(th, _fan_li(z, lam, O.SCAD_A), atol=1e-6)
