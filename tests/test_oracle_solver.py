"""Pins of the oracle's GD-PG solver (Algorithm 1, Sec. 3 and 5) against independent facts.

* lambda_max (Sec. 6.4): the solution is exactly zero at lambda_max and not below it;
* lambda = 0 Gaussian is weighted least squares (normal equations, np.linalg.lstsq);
* an orthonormal design has the closed-form lasso solution soft(X^T y, n lambda omega);
* the Gaussian lasso equals scikit-learn's coordinate-descent Lasso (independent solver);
* the Poisson, binomial and Gamma lassos equal L-BFGS-B on the split smooth reformulation
  (independent solver; its objective and gradient written from the densities, not the oracle);
* every lambda of a path meets the KKT conditions of Eq. (five);
* Thm. 1: the FISTA objective gap obeys 2 L ||x0 - x*||^2 / (l+1)^2;
* Thm. 2: F is nonincreasing over the outer iterations;
* the fixed point does not depend on the weights (Sec. 5, after the Corollary);
* the Gaussian family needs no line-search backtracking (Sec. 6.5: no outer loop);
* cells with observation weight 0 do not influence the fit (Sec. 4.3).
"""
import numpy as np
import pytest

import gen
import oracle as O


def _gauss(seed, n=(9, 7, 6), p=(4, 4, 4), pen="ones", mask=0.0):
    pr = gen.random_problem(seed, n, p, gen.GAUSSIAN, mask_frac=mask, basis="normal", pen_w=pen)
    return O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)


def _pois(seed, n=(8, 7, 6), p=(3, 3, 3), pen="ones", mask=0.0):
    pr = gen.random_problem(seed, n, p, gen.POISSON, mask_frac=mask, basis="normal", pen_w=pen)
    return O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)


def _binom(seed, n=(8, 7, 6), p=(3, 3, 3), pen="ones", mask=0.0):
    pr = gen.random_problem(seed, n, p, gen.BINOMIAL, mask_frac=mask, basis="normal", pen_w=pen)
    return O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)


def _gamma(seed, n=(8, 7, 6), p=(3, 3, 3), pen="ones", mask=0.0):
    pr = gen.random_problem(seed, n, p, gen.GAMMA, mask_frac=mask, basis="normal", pen_w=pen)
    return O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)


@pytest.mark.parametrize("maker", [_gauss, _pois, _binom, _gamma])
def test_lambda_max_zero_solution(maker):
    d = maker(20, pen="rand")
    lmax = O.lambda_max(d)
    th, st = O.gdpg(d, lmax, np.zeros(d.pshape), lmax, tol=1e-10)
    assert np.all(th == 0.0)
    th2, _ = O.gdpg(d, 0.99 * lmax, np.zeros(d.pshape), lmax, tol=1e-10)
    assert np.count_nonzero(th2) >= 1


def test_gaussian_lambda0_is_least_squares():
    d = _gauss(21, mask=0.2)
    lmax = O.lambda_max(d)
    th, st = O.gdpg(d, 0.0, np.zeros(d.pshape), lmax, tol=1e-11)
    Phi = O.kron_design(d.Xs)
    sw = np.sqrt(O.vec(d.a))
    ls, *_ = np.linalg.lstsq(sw[:, None] * Phi, sw * O.vec(d.Y), rcond=None)
    np.testing.assert_allclose(O.vec(th), ls, rtol=1e-7, atol=1e-9)


def test_orthonormal_closed_form():
    rng = np.random.default_rng(22)
    n, p = (6, 5, 4), (3, 3, 2)
    Xs = [np.linalg.qr(rng.standard_normal((n[j], p[j])))[0] for j in range(3)]
    Y = rng.standard_normal(n)
    pw = rng.uniform(0.5, 1.5, p)
    d = O.GlamData(O.GAUSSIAN, Xs, Y, np.ones(n), pw)
    Phi = np.kron(Xs[2], np.kron(Xs[1], Xs[0]))
    N = Y.size
    lmax = O.lambda_max(d)
    for lam in [0.7 * lmax, 0.3 * lmax, 0.05 * lmax]:
        th, _ = O.gdpg(d, lam, np.zeros(p), lmax, tol=1e-12)
        c = Phi.T @ O.vec(Y)
        closed = np.maximum(np.abs(c) - N * lam * O.vec(pw), 0) * np.sign(c)
        np.testing.assert_allclose(O.vec(th), closed, rtol=1e-10, atol=1e-12)


def test_gaussian_matches_sklearn_lasso():
    lm = pytest.importorskip("sklearn.linear_model")
    d = _gauss(23)
    Phi = O.kron_design(d.Xs)
    y = O.vec(d.Y)
    lams, thetas, stats, lmax = O.fit_path(d, nlambda=6, ratio=1e-2, tol=1e-11)
    for lam, th in zip(lams[1:], thetas[1:]):
        ref = lm.Lasso(alpha=lam, fit_intercept=False, tol=1e-14, max_iter=1_000_000).fit(Phi, y)
        np.testing.assert_allclose(O.vec(th), ref.coef_, rtol=1e-6, atol=1e-8)
        assert set(np.flatnonzero(O.vec(th))) == set(np.flatnonzero(ref.coef_))


def test_poisson_matches_lbfgsb_split_form():
    from scipy.optimize import minimize
    d = _pois(24, pen="rand", mask=0.15)
    Phi = O.kron_design(d.Xs)
    y, a, w = O.vec(d.Y), O.vec(d.a), O.vec(d.pen_w)
    N, P = Phi.shape
    lmax = O.lambda_max(d)
    lam = 0.2 * lmax

    def fg(v):
        th = v[:P] - v[P:]
        eta = Phi @ th
        mu = np.exp(eta)
        f = np.sum(a * (mu - y * eta)) / N + lam * np.sum(w * (v[:P] + v[P:]))
        g = Phi.T @ (a * (mu - y)) / N
        return f, np.concatenate([g + lam * w, -g + lam * w])

    res = minimize(fg, np.zeros(2 * P), jac=True, method="L-BFGS-B", bounds=[(0, None)] * (2 * P),
                   options={"ftol": 1e-16, "gtol": 1e-13, "maxiter": 100000, "maxcor": 30})
    ref = res.x[:P] - res.x[P:]
    th, st = O.gdpg(d, lam, np.zeros(d.pshape), lmax, tol=1e-11)
    assert st.converged
    F_or = O.objective(d, th, lam)
    assert F_or <= res.fun + 1e-12
    np.testing.assert_allclose(O.vec(th), ref, atol=2e-5)


def _nll_and_grad(family, eta, y, a):
    """sum_i a_i l_i and d/deta from the densities themselves (Bernoulli-trial proportions with
    a_i trials; exponential with mean exp(eta))."""
    if family == gen.BINOMIAL:
        mu = 1.0 / (1.0 + np.exp(-eta))
        return np.sum(a * (np.logaddexp(0.0, eta) - y * eta)), a * (mu - y)
    if family == gen.GAMMA:
        return np.sum(a * (y * np.exp(-eta) + eta)), a * (1.0 - y * np.exp(-eta))
    mu = np.exp(eta)
    return np.sum(a * (mu - y * eta)), a * (mu - y)


@pytest.mark.parametrize("maker", [_binom, _gamma])
def test_binomial_and_gamma_match_lbfgsb_split_form(maker):
    from scipy.optimize import minimize
    d = maker(26, pen="rand", mask=0.15)
    Phi = O.kron_design(d.Xs)
    y, a, w = O.vec(d.Y), O.vec(d.a), O.vec(d.pen_w)
    N, P = Phi.shape
    lmax = O.lambda_max(d)
    lam = 0.2 * lmax

    def fg(v):
        th = v[:P] - v[P:]
        f, ge = _nll_and_grad(d.family, Phi @ th, y, a)
        g = Phi.T @ ge / N
        return f / N + lam * np.sum(w * (v[:P] + v[P:])), np.concatenate([g + lam * w, -g + lam * w])

    res = minimize(fg, np.zeros(2 * P), jac=True, method="L-BFGS-B", bounds=[(0, None)] * (2 * P),
                   options={"ftol": 1e-16, "gtol": 1e-13, "maxiter": 100000, "maxcor": 30})
    ref = res.x[:P] - res.x[P:]
    # (the Fisher weight of the Gamma log link understates the curvature where y > mu, so the
    # line search backtracks often and the last digits come slowly: KKT 1e-10 there)
    th, st = O.gdpg(d, lam, np.zeros(d.pshape), lmax, tol=1e-10 if d.family == gen.GAMMA else 1e-11)
    assert st.converged
    # the objectives differ by the dropped constants only: compare through the same function
    F_or = fg(np.concatenate([np.maximum(O.vec(th), 0), np.maximum(-O.vec(th), 0)]))[0]
    assert F_or <= res.fun + 1e-12
    np.testing.assert_allclose(O.vec(th), ref, atol=2e-5)


@pytest.mark.parametrize("maker", [_gauss, _pois, _binom, _gamma])
def test_path_meets_kkt(maker):
    d = maker(25, pen="rand", mask=0.1)
    lams, thetas, stats, lmax = O.fit_path(d, nlambda=5, ratio=1e-2, tol=1e-9)
    for lam, th, st in zip(lams, thetas, stats):
        assert st.converged
        assert O.kkt_residual(d, th, lam, lmax) <= 1e-9
    nnz = [np.count_nonzero(t) for t in thetas]
    assert nnz[0] == 0 and nnz[-1] > 0


def test_thm1_fista_rate():
    d = _gauss(26)                       # W = 1, so L_hat = L exactly
    lmax = O.lambda_max(d)
    lam = 0.1 * lmax
    w = d.a.copy()
    z = d.Y.copy()
    L = O.lipschitz_exact(d.Xs, w)
    assert np.isclose(L, O.lipschitz_bound(d.Xs, w), rtol=1e-10)
    x0 = np.zeros(d.pshape)
    star = O.inner_pg(d, w, z, x0, 1.0 / L, lam, tol=1e-15, max_iter=200000).x
    run = O.inner_pg(d, w, z, x0, 1.0 / L, lam, tol=0.0, max_iter=300, keep_history=True)

    def Gobj(x):   # h + lambda J with h of Eq. (twentyfour)
        r = O.H(d.Xs, x) - z
        return float(np.sum(w * r * r)) / (2 * d.n) + lam * O.penalty(x, d.pen_w)

    G_star = Gobj(star)
    R2 = float(np.sum((x0 - star) ** 2))
    for l in range(1, 300):
        gap = Gobj(run.history[l - 1]) - G_star    # history[l-1] is x(l)
        assert gap <= 2 * L * R2 / (l + 1) ** 2 + 1e-13


def test_thm2_monotone_objective():
    d = _pois(27, mask=0.1)
    lmax = O.lambda_max(d)
    th, st = O.gdpg(d, 0.05 * lmax, np.zeros(d.pshape), lmax, tol=1e-10, tol_inner=1e-6)
    tr = np.array(st.objective_trace)
    assert len(tr) >= 3
    assert np.all(np.diff(tr) <= 1e-14)


def test_fixed_point_independent_of_weights():
    d = _pois(28, mask=0.1)
    lmax = O.lambda_max(d)
    lam = 0.1 * lmax
    a, _ = O.gdpg(d, lam, np.zeros(d.pshape), lmax, tol=1e-11, weights="exact")
    b, _ = O.gdpg(d, lam, np.zeros(d.pshape), lmax, tol=1e-11, weights="one")
    np.testing.assert_allclose(a, b, atol=1e-7)
    assert set(np.flatnonzero(a)) == set(np.flatnonzero(b))


def test_gaussian_has_no_line_search():
    d = _gauss(29, mask=0.2)
    lams, thetas, stats, lmax = O.fit_path(d, nlambda=4, ratio=1e-2, tol=1e-9)
    assert all(st.armijo_backtracks == 0 for st in stats)


def test_masked_cells_do_not_matter():
    d = _pois(30, mask=0.3)
    lmax = O.lambda_max(d)
    th1, _ = O.gdpg(d, 0.1 * lmax, np.zeros(d.pshape), lmax, tol=1e-10)
    Y2 = d.Y.copy(order="K")   # same memory order, so every sum runs in the same order
    Y2[d.a == 0] = 123.0
    d2 = O.GlamData(d.family, d.Xs, Y2, d.a, d.pen_w)
    assert O.lambda_max(d2) == lmax
    th2, _ = O.gdpg(d2, 0.1 * lmax, np.zeros(d.pshape), lmax, tol=1e-10)
    np.testing.assert_array_equal(th1, th2)


def test_planted_sign_slip_is_caught(monkeypatch):
    """A sign slip in the score (a plausible mistake) breaks the KKT pin of the path."""
    d = _gauss(31)
    lmax = O.lambda_max(d)
    th, _ = O.gdpg(d, 0.2 * lmax, np.zeros(d.pshape), lmax, tol=1e-10)
    good = O.glam_oracle.score
    monkeypatch.setattr(O.glam_oracle, "score", lambda f, e, y, a: -good(f, e, y, a))
    assert O.glam_oracle.kkt_residual(d, th, 0.2 * lmax, lmax) > 1e-3
