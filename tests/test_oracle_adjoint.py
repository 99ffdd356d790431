"""Pins of the oracle's derivatives used by the adjoint (autograd) check.

* df/dy (`loss_grad_y`) against central finite differences of the loss in y, which is exact up
  to rounding because f is linear (Poisson) or quadratic (Gaussian) in y;
* the penalized gradient (`penalized_gradient`) against central finite differences of the
  objective F of Eq. (five) along coordinates away from the kink of |theta_m|, and against
  random directions that leave the zero coordinates alone;
* a planted mistake (a dropped observation weight in df/dy) is caught by the same check.
"""
import numpy as np
import pytest

import oracle as O


def _data(rng, fam, n=(6, 5, 4), p=(4, 3, 3)):
    Xs = [rng.standard_normal((n[j], p[j])) * 0.5 for j in range(3)]
    theta = rng.standard_normal(p) * 0.4
    theta[rng.random(p) < 0.3] = 0.0
    eta = O.H(Xs, theta)
    if fam == O.GAUSSIAN:
        y = eta + rng.standard_normal(n)
    else:
        y = rng.poisson(np.exp(eta)).astype(float)
    a = rng.uniform(0.5, 2.0, n)
    a[rng.random(n) < 0.2] = 0.0
    pw = rng.uniform(0.5, 1.5, p)
    return O.GlamData(fam, Xs, y, a, pw), theta


@pytest.mark.parametrize("fam", [O.GAUSSIAN, O.POISSON])
def test_loss_grad_y_matches_finite_differences(fam):
    rng = np.random.default_rng(40 + fam)
    d, theta = _data(rng, fam)
    eta = O.H(d.Xs, theta)
    g = O.loss_grad_y(fam, eta, d.Y, d.a)
    h = 1e-3
    for _ in range(5):
        D = rng.standard_normal(d.Y.shape)
        fd = (O.loss(fam, eta, d.Y + h * D, d.a) - O.loss(fam, eta, d.Y - h * D, d.a)) / (2 * h)
        assert abs(fd - float(np.sum(g * D))) <= 1e-10 * (1 + abs(fd))


@pytest.mark.parametrize("fam", [O.GAUSSIAN, O.POISSON])
def test_penalized_gradient_matches_finite_differences(fam):
    rng = np.random.default_rng(50 + fam)
    d, theta = _data(rng, fam)
    lam = 0.3 * O.lambda_max(d)
    g = O.penalized_gradient(d, theta, lam)
    h = 1e-5
    for m in zip(*np.nonzero(np.abs(theta) > 2 * h)):
        e = np.zeros_like(theta)
        e[m] = 1.0
        fd = (O.objective(d, theta + h * e, lam) - O.objective(d, theta - h * e, lam)) / (2 * h)
        assert abs(fd - g[m]) <= 1e-7 * (1 + abs(g[m]))
    # directions that leave the zero coordinates (the kinks) untouched
    for _ in range(4):
        D = rng.standard_normal(theta.shape) * (np.abs(theta) > 2 * h)
        fd = (O.objective(d, theta + h * D, lam) - O.objective(d, theta - h * D, lam)) / (2 * h)
        assert abs(fd - float(np.sum(g * D))) <= 1e-7 * (1 + np.linalg.norm(g) * np.linalg.norm(D))


def test_penalized_gradient_zero_coordinates_use_sign_zero():
    rng = np.random.default_rng(60)
    d, theta = _data(rng, O.POISSON)
    lam = 0.5
    g = O.penalized_gradient(d, theta, lam)
    zero = theta == 0
    assert zero.any()
    assert np.array_equal(g[zero], O.gradient(d, theta)[zero])


def test_planted_dropped_weight_in_grad_y_is_caught():
    rng = np.random.default_rng(70)
    d, theta = _data(rng, O.POISSON)
    eta = O.H(d.Xs, theta)
    wrong = -eta / d.n  # the observation weight a_i left out
    h = 1e-3
    D = rng.standard_normal(d.Y.shape)
    fd = (O.loss(O.POISSON, eta, d.Y + h * D, d.a) - O.loss(O.POISSON, eta, d.Y - h * D, d.a)) / (2 * h)
    assert abs(fd - float(np.sum(wrong * D))) > 1e-6
