"""Pins of the oracle's family quantities (App. B), prox (Sec. 6.3) and step size (Prop. 1).

* the loss is the negative log-likelihood of scipy's Gaussian / Poisson densities up to the
  stated constants;
* the score is u = dl/deta (finite differences), the IRLS weight of a canonical link is
  w = -du/deta (finite differences);
* the working response makes the quadratic model h of Eq. (twentyfour) a second-order
  model of f at the anchor: grad h(theta_k) = grad f(theta_k) and the Hessians agree;
* the soft threshold is the minimiser of (1/2)(x - z)^2 + gamma |x| (brute force);
* L <= L_hat (Prop. 1) with equality when W = c I.
"""
import numpy as np
import pytest

import oracle as O

scipy_stats = pytest.importorskip("scipy.stats")


def _data(rng, fam, n=(5, 4, 3), p=(3, 2, 3), mask=False):
    Xs = [rng.standard_normal((n[j], p[j])) * 0.5 for j in range(3)]
    eta = rng.uniform(-1.5, 1.5, n)
    if fam == O.GAUSSIAN:
        y = eta + rng.standard_normal(n)
    elif fam == O.POISSON:
        y = rng.poisson(np.exp(eta)).astype(float)
    elif fam == O.BINOMIAL:
        y = rng.binomial(6, 1.0 / (1.0 + np.exp(-eta))) / 6.0
    else:
        y = rng.gamma(2.0, np.exp(eta) / 2.0)
    a = rng.uniform(0.5, 2.0, n)
    if mask:
        a[rng.random(n) < 0.3] = 0.0
    pw = rng.uniform(0.5, 1.5, p)
    return O.GlamData(fam, Xs, y, a, pw), eta


def test_poisson_loss_is_negative_loglik():
    rng = np.random.default_rng(10)
    d, eta = _data(rng, O.POISSON)
    logpmf = scipy_stats.poisson.logpmf(d.Y, np.exp(eta))
    from scipy.special import gammaln
    expected = -np.sum(d.a * (logpmf + gammaln(d.Y + 1))) / d.n
    assert np.isclose(O.loss(O.POISSON, eta, d.Y, d.a), expected, rtol=1e-13)


def test_gaussian_loss_is_negative_loglik():
    rng = np.random.default_rng(11)
    d, eta = _data(rng, O.GAUSSIAN)
    logpdf = scipy_stats.norm.logpdf(d.Y, loc=eta, scale=1.0)
    expected = -np.sum(d.a * (logpdf + 0.5 * np.log(2 * np.pi))) / d.n
    assert np.isclose(O.loss(O.GAUSSIAN, eta, d.Y, d.a), expected, rtol=1e-13)


ALL = [O.GAUSSIAN, O.POISSON, O.BINOMIAL, O.GAMMA]


@pytest.mark.parametrize("fam", ALL)
def test_score_is_derivative_of_loglik(fam):
    rng = np.random.default_rng(12)
    d, eta = _data(rng, fam, mask=True)
    u = O.score(fam, eta, d.Y, d.a)
    h = 1e-6
    for idx in [(0, 0, 0), (4, 3, 2), (2, 1, 1)]:
        e1, e2 = eta.copy(), eta.copy()
        e1[idx] += h
        e2[idx] -= h
        fd = (O.loglik(fam, e1, d.Y, d.a) - O.loglik(fam, e2, d.Y, d.a)) / (2 * h)
        assert np.isclose(u[idx], fd, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("fam", ALL)
def test_weight_is_fisher_information(fam):
    """w = E[-du/deta]: -du/deta with y replaced by its mean g^{-1}(eta) (for a canonical link
    du/deta does not depend on y at all)."""
    rng = np.random.default_rng(13)
    d, eta = _data(rng, fam, mask=True)
    w = O.irls_weight(fam, eta, d.a)
    h = 1e-6
    mu = O.mean_response(fam, eta)
    du = (O.score(fam, eta + h, mu, d.a) - O.score(fam, eta - h, mu, d.a)) / (2 * h)
    np.testing.assert_allclose(w, -du, rtol=1e-6, atol=1e-9)
    assert np.all(w[d.a == 0] == 0) and np.all(w[d.a > 0] > 0)


@pytest.mark.parametrize("fam", ALL)
def test_quadratic_model_matches_f_to_second_order(fam):
    """grad h = grad f at the anchor; the Hessians agree where the Fisher weight is the observed
    curvature: always for a canonical link, and for the Gamma family's log link where y equals
    its mean at the anchor (the data are set so)."""
    rng = np.random.default_rng(14)
    d, _ = _data(rng, fam, mask=True)
    theta_k = rng.standard_normal(d.pshape) * 0.2
    eta_k = O.H(d.Xs, theta_k)
    if fam == O.GAMMA:
        d = O.GlamData(fam, d.Xs, O.mean_response(fam, eta_k), d.a, d.pen_w)
    w = O.irls_weight(fam, eta_k, d.a)
    z = O.working_response(fam, eta_k, d.Y, d.a)

    def grad_h(theta):  # Eq. (twentyfive), explicit design
        Phi = O.kron_design(d.Xs)
        return O.unvec(Phi.T @ (O.vec(w) * (Phi @ O.vec(theta) - O.vec(z))) / d.n, d.pshape)

    np.testing.assert_allclose(grad_h(theta_k), O.gradient(d, theta_k), rtol=1e-10, atol=1e-12)
    # Hessian-vector products: d/dt grad f(theta + t v) at t = 0 == X^T W X v / n
    v = rng.standard_normal(d.pshape)
    t = 1e-5
    hv_f = (O.gradient(d, theta_k + t * v) - O.gradient(d, theta_k - t * v)) / (2 * t)
    hv_h = grad_h(theta_k + v) - grad_h(theta_k)
    np.testing.assert_allclose(hv_f, hv_h, rtol=1e-6, atol=1e-9)
    # masked cells: z = eta
    np.testing.assert_array_equal(z[d.a == 0], eta_k[d.a == 0])


def test_soft_threshold_is_prox():
    from scipy.optimize import minimize_scalar
    rng = np.random.default_rng(15)
    for z, g in zip(rng.standard_normal(40) * 2, rng.uniform(0, 1.5, 40)):
        res = minimize_scalar(lambda x: 0.5 * (x - z) ** 2 + g * abs(x), bounds=(-10, 10),
                              method="bounded", options={"xatol": 1e-12})
        assert abs(O.soft_threshold(np.array([z]), g)[0] - res.x) < 1e-6
    # ties: |z| == gamma gives exactly zero
    assert O.soft_threshold(np.array([0.5, -0.5]), 0.5).tolist() == [0.0, 0.0]


def test_prop1_bound():
    rng = np.random.default_rng(16)
    n, p = (6, 5, 4), (3, 4, 3)
    Xs = [rng.standard_normal((n[j], p[j])) for j in range(3)]
    for _ in range(3):
        w = rng.uniform(0.1, 3.0, n)
        L = O.lipschitz_exact(Xs, w)
        Lh = O.lipschitz_bound(Xs, w)
        assert L <= Lh * (1 + 1e-12)
        # power iteration on the explicit X^T W X / n (independent of eigvalsh)
        Phi = O.kron_design(Xs)
        M = Phi.T @ (O.vec(w)[:, None] * Phi) / Phi.shape[0]
        x = np.ones(M.shape[0])
        for _ in range(3000):
            x = M @ x
            x /= np.linalg.norm(x)
        assert x @ M @ x <= Lh * (1 + 1e-12)
    # W = c I: the bound is exact (spectral radius of a Kronecker product is the product)
    w = np.full(n, 2.5)
    assert np.isclose(O.lipschitz_exact(Xs, w), O.lipschitz_bound(Xs, w), rtol=1e-10)


def test_binomial_loss_is_negative_loglik():
    rng = np.random.default_rng(15)
    m = rng.integers(1, 9, (5, 4, 3))
    eta = rng.uniform(-2, 2, m.shape)
    k = rng.binomial(m, 1.0 / (1.0 + np.exp(-eta)))
    y, a = k / m, m.astype(float)
    logpmf = scipy_stats.binom.logpmf(k, m, 1.0 / (1.0 + np.exp(-eta)))
    from scipy.special import comb
    expected = -np.sum(logpmf - np.log(comb(m, k))) / eta.size
    assert np.isclose(O.loss(O.BINOMIAL, eta, y, a), expected, rtol=1e-12)


def test_gamma_loss_is_negative_loglik():
    """Dispersion 1 (shape 1): the exponential density with mean exp(eta)."""
    rng = np.random.default_rng(16)
    eta = rng.uniform(-1, 2, (5, 4, 3))
    y = rng.exponential(np.exp(eta))
    a = rng.uniform(0.5, 2.0, eta.shape)
    logpdf = scipy_stats.expon.logpdf(y, scale=np.exp(eta))
    assert np.isclose(O.loss(O.GAMMA, eta, y, a), -np.sum(a * logpdf) / eta.size, rtol=1e-12)


def test_planted_gamma_canonical_slip_is_caught():
    """Treating the Gamma log link as canonical (theta'(eta) = 1) breaks the score pin."""
    rng = np.random.default_rng(17)
    d, eta = _data(rng, O.GAMMA)
    wrong = d.a * (d.Y - np.exp(eta))
    h = 1e-6
    e1, e2 = eta.copy(), eta.copy()
    e1[0, 0, 0] += h
    e2[0, 0, 0] -= h
    fd = (O.loglik(O.GAMMA, e1, d.Y, d.a) - O.loglik(O.GAMMA, e2, d.Y, d.a)) / (2 * h)
    assert not np.isclose(wrong[0, 0, 0], fd, rtol=1e-3)
