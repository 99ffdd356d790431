"""Pins of the oracle's model with c > 1 components (Sec. 2, Eq. fivenew: X = [X_1 | ... | X_c];
Eqs. eighteen/nineteen with r = 1..c; Prop. 1, Eq. nineteennew, with the sum over r).

* H and G with components equal the explicit concatenated design X theta and X^T vec(U) (tiny
  sizes; each block the np.kron tensor product of its component's designs);
* one component given as a component list is the plain model;
* the Prop. 1 factor sum_r prod_j varrho(X_rj^T X_rj) is not below varrho(X^T X) of the
  concatenated design;
* the Gaussian lasso path with two components equals scikit-learn's Lasso on the explicit
  concatenated design, and a Poisson fit with two components meets its KKT conditions, which the
  explicit design confirms;
* a planted mistake (the second component's block of G left out) is caught.
"""
import numpy as np
import pytest

import oracle as O


def _comps(seed, n=(6, 5, 4), ps=((3, 2, 2), (2, 3, 1))):
    rng = np.random.default_rng(seed)
    comps = [[rng.standard_normal((n[j], p[j])) for j in range(3)] for p in ps]
    return rng, comps


def _explicit(comps):
    return np.hstack([O.kron_design(Xr) for Xr in comps])


def test_components_H_and_G_equal_explicit_design():
    rng, comps = _comps(1)
    n = tuple(X.shape[0] for X in comps[0])
    Phi = _explicit(comps)
    d = O.GlamData(O.GAUSSIAN, comps[0], np.zeros(n), np.ones(n), np.ones(Phi.shape[1]), comps=comps)
    theta = rng.standard_normal(Phi.shape[1])
    assert d.pshape == (Phi.shape[1],)
    np.testing.assert_allclose(O.vec(d.H(theta)), Phi @ theta, rtol=1e-13, atol=1e-13)
    U = rng.standard_normal(n)
    np.testing.assert_allclose(d.G(U), Phi.T @ O.vec(U), rtol=1e-13, atol=1e-13)


def test_single_component_list_is_the_plain_model():
    rng, comps = _comps(2, ps=((3, 2, 2),))
    n = tuple(X.shape[0] for X in comps[0])
    p = tuple(X.shape[1] for X in comps[0])
    a = O.GlamData(O.POISSON, comps[0], np.ones(n), np.ones(n), np.ones(p))
    b = O.GlamData(O.POISSON, comps[0], np.ones(n), np.ones(n), np.ones(int(np.prod(p))), comps=comps)
    theta = rng.standard_normal(p)
    np.testing.assert_allclose(O.vec(a.H(theta)), O.vec(b.H(O.vec(theta))), rtol=1e-14)
    U = rng.standard_normal(n)
    np.testing.assert_allclose(O.vec(a.G(U)), b.G(U), rtol=1e-14)
    assert a.rho_sum() == pytest.approx(b.rho_sum(), rel=1e-14)


def test_prop1_factor_bounds_concatenated_design():
    for seed in range(5):
        _, comps = _comps(10 + seed)
        n = tuple(X.shape[0] for X in comps[0])
        Phi = _explicit(comps)
        d = O.GlamData(O.GAUSSIAN, comps[0], np.zeros(n), np.ones(n), np.ones(Phi.shape[1]), comps=comps)
        exact = float(np.max(np.linalg.eigvalsh(Phi.T @ Phi)))
        assert d.rho_sum() >= exact * (1 - 1e-12)


def _gauss_components(seed):
    rng, comps = _comps(seed, n=(7, 6, 5))
    Phi = _explicit(comps)
    n = tuple(X.shape[0] for X in comps[0])
    th = rng.standard_normal(Phi.shape[1]) * (rng.random(Phi.shape[1]) < 0.5)
    y = Phi @ th + 0.3 * rng.standard_normal(Phi.shape[0])
    Y = O.unvec(y, n)
    return O.GlamData(O.GAUSSIAN, comps[0], Y, np.ones(n), np.ones(Phi.shape[1]), comps=comps), Phi


def test_two_component_gaussian_lasso_matches_sklearn():
    lm = pytest.importorskip("sklearn.linear_model")
    d, Phi = _gauss_components(21)
    lams, thetas, stats, lmax = O.fit_path(d, nlambda=5, ratio=1e-2, tol=1e-11)
    y = O.vec(d.Y)
    for lam, th in zip(lams[1:], thetas[1:]):
        ref = lm.Lasso(alpha=lam, fit_intercept=False, tol=1e-14, max_iter=1_000_000).fit(Phi, y)
        np.testing.assert_allclose(th, ref.coef_, rtol=1e-6, atol=1e-8)


def test_two_component_poisson_fit_meets_kkt_by_explicit_design():
    rng, comps = _comps(22, n=(7, 6, 5))
    Phi = _explicit(comps)
    n = tuple(X.shape[0] for X in comps[0])
    eta = 0.3 * (Phi @ (0.5 * rng.standard_normal(Phi.shape[1])))
    Y = O.unvec(rng.poisson(np.exp(eta)).astype(np.float64), n)
    a = np.ones(n)
    a.reshape(-1)[rng.choice(a.size, 20, replace=False)] = 0.0
    pw = rng.uniform(0.5, 1.5, Phi.shape[1])
    d = O.GlamData(O.POISSON, comps[0], Y, a, pw, comps=comps)
    lmax = O.lambda_max(d)
    lam = 0.1 * lmax
    th, st = O.gdpg(d, lam, np.zeros(Phi.shape[1]), lmax, tol=1e-10)
    assert st.converged
    # the KKT residual recomputed with the explicit design and the score of App. B
    eta_e = O.unvec(Phi @ th, n)
    g = -(Phi.T @ O.vec(O.score(O.POISSON, eta_e, Y, a))) / eta_e.size
    r = np.where(th != 0, np.abs(g + lam * pw * np.sign(th)), np.maximum(0.0, np.abs(g) - lam * pw))
    assert float(np.max(r)) / lmax <= 1e-9


def test_planted_missing_component_block_is_caught():
    rng, comps = _comps(3)
    n = tuple(X.shape[0] for X in comps[0])
    Phi = _explicit(comps)
    d = O.GlamData(O.GAUSSIAN, comps[0], np.zeros(n), np.ones(n), np.ones(Phi.shape[1]), comps=comps)
    U = rng.standard_normal(n)
    good = d.G(U)
    k0 = O.kron_design(comps[0]).shape[1]
    planted = np.concatenate([good[:k0], np.zeros(good.size - k0)])
    assert not np.allclose(planted, Phi.T @ O.vec(U), rtol=1e-6)
