"""Pins of the oracle's elastic-net and ridge penalties (Sec. 6.3).

* the prox is the minimiser of (1/2)(x - z)^2 + gamma (l1 |x| + l2 x^2) (brute force on a grid
  refined around the candidates);
* the ridge fit of a Gaussian model is the solution of the regularised normal equations
  (X^T W X / n + 2 lambda diag(omega)) theta = X^T W y / n (linear algebra on the explicit design);
* the elastic net equals L-BFGS-B on the split smooth form (Poisson family);
* the elastic net at l2 = 0 is the lasso;
* a planted mistake in the prox (the ridge factor without its 2) is caught.
"""
import numpy as np
import pytest

import gen
import oracle as O


def test_prox_is_the_minimiser():
    rng = np.random.default_rng(80)
    for l1, l2 in [(1.0, 0.0), (1.0, 0.7), (0.0, 1.0), (1.0, 3.0)]:
        for _ in range(20):
            z, gam = rng.normal(0, 2), rng.uniform(0.05, 1.5)
            xs = np.linspace(-6, 6, 240001)
            obj = 0.5 * (xs - z) ** 2 + gam * (l1 * np.abs(xs) + l2 * xs * xs)
            ref = xs[np.argmin(obj)]
            assert abs(O.penalty_prox(np.array(z), gam, l1, l2) - ref) <= 1e-4


def _gauss(seed, l1, l2, mask=0.1):
    pr = gen.random_problem(seed, (9, 7, 6), (4, 4, 3), gen.GAUSSIAN, mask_frac=mask, basis="normal",
                            pen_w="rand")
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    return O.GlamData(d.family, d.Xs, d.Y, d.a, d.pen_w, l1, l2)


def test_ridge_is_regularised_least_squares():
    d = _gauss(81, 0.0, 1.0)
    lmax = O.lambda_max(d)
    lam = 0.05 * lmax
    th, st = O.gdpg(d, lam, np.zeros(d.pshape), lmax, tol=1e-11)
    assert st.converged
    Phi = O.kron_design(d.Xs)
    a, y, w = O.vec(d.a), O.vec(d.Y), O.vec(d.pen_w)
    A = Phi.T @ (a[:, None] * Phi) / d.n + 2.0 * lam * np.diag(w)
    ref = np.linalg.solve(A, Phi.T @ (a * y) / d.n)
    np.testing.assert_allclose(O.vec(th), ref, rtol=1e-8, atol=1e-10)


def test_enet_zero_l2_is_the_lasso():
    d = _gauss(82, 1.0, 0.0)
    lmax = O.lambda_max(d)
    dl = O.GlamData(d.family, d.Xs, d.Y, d.a, d.pen_w)
    a, _ = O.gdpg(d, 0.2 * lmax, np.zeros(d.pshape), lmax, tol=1e-11)
    b, _ = O.gdpg(dl, 0.2 * lmax, np.zeros(d.pshape), lmax, tol=1e-11)
    np.testing.assert_array_equal(a, b)


def test_poisson_enet_matches_lbfgsb_split_form():
    from scipy.optimize import minimize
    pr = gen.random_problem(83, (8, 7, 6), (3, 3, 3), gen.POISSON, mask_frac=0.1, basis="normal",
                            pen_w="rand")
    d0 = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    l2 = 0.8
    d = O.GlamData(d0.family, d0.Xs, d0.Y, d0.a, d0.pen_w, 1.0, l2)
    Phi = O.kron_design(d.Xs)
    y, a, w = O.vec(d.Y), O.vec(d.a), O.vec(d.pen_w)
    N, P = Phi.shape
    lmax = O.lambda_max(d)
    lam = 0.15 * lmax

    def fg(v):
        th = v[:P] - v[P:]
        eta = Phi @ th
        mu = np.exp(eta)
        f = (np.sum(a * (mu - y * eta)) / N + lam * np.sum(w * (v[:P] + v[P:]))
             + lam * l2 * np.sum(w * th * th))
        g = Phi.T @ (a * (mu - y)) / N + 2.0 * lam * l2 * w * th
        return f, np.concatenate([g + lam * w, -g + lam * w])

    res = minimize(fg, np.zeros(2 * P), jac=True, method="L-BFGS-B", bounds=[(0, None)] * (2 * P),
                   options={"ftol": 1e-16, "gtol": 1e-13, "maxiter": 100000, "maxcor": 30})
    th, st = O.gdpg(d, lam, np.zeros(d.pshape), lmax, tol=1e-11)
    assert st.converged
    np.testing.assert_allclose(O.vec(th), res.x[:P] - res.x[P:], atol=2e-5)
    assert O.objective(d, th, lam) <= res.fun + 1e-12


def test_planted_ridge_factor_slip_is_caught(monkeypatch):
    d = _gauss(81, 0.0, 1.0)
    lmax = O.lambda_max(d)
    lam = 0.05 * lmax
    good = O.glam_oracle.soft_threshold
    monkeypatch.setattr(O.glam_oracle, "penalty_prox",
                        lambda z, g, l1=1.0, l2=0.0: good(z, g * l1) / (1.0 + g * l2))
    th, _ = O.glam_oracle.gdpg(d, lam, np.zeros(d.pshape), lmax, tol=1e-11, max_outer=20)
    Phi = O.kron_design(d.Xs)
    a, y, w = O.vec(d.a), O.vec(d.Y), O.vec(d.pen_w)
    A = Phi.T @ (a[:, None] * Phi) / d.n + 2.0 * lam * np.diag(w)
    ref = np.linalg.solve(A, Phi.T @ (a * y) / d.n)
    assert not np.allclose(O.vec(th), ref, rtol=1e-6, atol=1e-8)
