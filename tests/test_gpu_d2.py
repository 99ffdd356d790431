"""Plans of a 2-D GLAM (d = 2: n3 = p3 = 1, X3 = [1], passed as None) against the oracle, with one
component.  The model is Eq. (fivenew) with a design of two factors; Sec. 6.4 lists d = 2 and 3.

* glam_predict, glam_gradient and glam_loss, all four families, FP64 and FP32 plans, element by
  element against the absolute-value chains, at a ragged shape (37 x 29) and at a shape of the
  tensor-core kernels (128 x 96, where an FP32 plan's inner loop runs on tcgen05 with one slab);
* glam_fit_path (Gaussian, masked Poisson; FP64 and FP32 plans) reaches the oracle's solutions:
  the oracle's KKT residual at every returned lambda, and at the ragged shape the objectives of
  the oracle's own path.
"""
import numpy as np
import pytest

import gen
import oracle as O
from gpu_helpers import BAR, assert_within, cell_scales, chain_G, chain_H, dev, dtype_of, gpu_or_skip, host, \
    plan_prec

pytestmark = pytest.mark.gpu

SHAPES = [((37, 29), (9, 7)), ((128, 96), (24, 20))]


def _problem(seed, n, p, fam, mask=0.1):
    """N(0, 1/n_j) designs in modes 1 and 2, X3 = [1], a sparse truth and the family's response;
    C layout (XT[j] (p_j, n_j); Y, W and the coefficients (1, n2, n1) / (1, p2, p1))."""
    rng = np.random.default_rng(seed)
    XT = [rng.standard_normal((p[j], n[j])) / np.sqrt(n[j]) for j in range(2)] + [np.ones((1, 1))]
    truth = rng.standard_normal((1, p[1], p[0])) * (rng.random((1, p[1], p[0])) < 0.4)
    eta = O.predict_c(XT, truth)
    W = np.ones(eta.shape)
    if fam == gen.GAUSSIAN:
        Y = eta + 0.3 * rng.standard_normal(eta.shape)
    else:
        eta = 1.5 * np.tanh(eta)
        if fam == gen.POISSON:
            Y = rng.poisson(np.exp(eta)).astype(np.float64)
        elif fam == gen.BINOMIAL:
            m = rng.integers(1, 9, eta.shape)
            Y = rng.binomial(m, 1.0 / (1.0 + np.exp(-eta))) / m
            W = m.astype(np.float64)
        else:
            Y = rng.gamma(2.0, np.exp(eta) / 2.0)
    W.reshape(-1)[rng.choice(W.size, int(mask * W.size), replace=False)] = 0.0
    pen = rng.uniform(0.5, 1.5, (1, p[1], p[0]))
    return XT, Y, W, pen


def _cast(prec, a):
    return np.asarray(a, np.float64) if prec == "fp64" else np.asarray(a, np.float32).astype(np.float64)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON, gen.BINOMIAL, gen.GAMMA])
@pytest.mark.parametrize("n,p", SHAPES)
def test_d2_predict_gradient_loss_match_oracle(prec, fam, n, p):
    torch, g = gpu_or_skip()
    XT, Y, W, pen = _problem(71, n, p, fam)
    XT, Y, W = [_cast(prec, x) for x in XT], _cast(prec, Y), _cast(prec, W)
    d = O.GlamData.from_c(fam, XT, Y, W, pen)
    dt = dtype_of(prec)
    plan = g.Plan(n, p, fam, plan_prec(g, prec))
    X = [dev(x, dt) for x in XT[:2]] + [None]
    theta = _cast(prec, 0.3 * np.random.default_rng(72).standard_normal((1, p[1], p[0])))
    th = O.paper_array(theta)
    eta_abs = chain_H(d.Xs, th)
    eta = g.glam_predict(plan, X, dev(theta, dt))
    assert_within(host(eta), O.predict_c(XT, theta), O.c_array(eta_abs), BAR[prec], what="eta")
    grad, loss = g.glam_gradient(plan, X, dev(theta, dt), dev(Y, dt), dev(W, dt), want_loss=True)
    su, _, _ = cell_scales(fam, O.H(d.Xs, th), eta_abs, d.Y, d.a)
    assert_within(host(grad), O.c_array(O.gradient(d, th)), O.c_array(chain_G(d.Xs, su)) / d.n, BAR[prec],
                  what="grad")
    fref = O.loss(fam, O.H(d.Xs, th), d.Y, d.a)
    assert abs(loss.item() - fref) <= (1e-12 if prec == "fp64" else 1e-6) * abs(fref)
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON])
@pytest.mark.parametrize("n,p", SHAPES)
def test_d2_fit_path_matches_oracle(prec, fam, n, p):
    torch, g = gpu_or_skip()
    XT, Y, W, pen = _problem(73, n, p, fam, mask=0.1 if fam == gen.POISSON else 0.0)
    XT, Y, W = [_cast(prec, x) for x in XT], _cast(prec, Y), _cast(prec, W)
    d = O.GlamData.from_c(fam, XT, Y, W, pen)
    lmax = O.lambda_max(d)
    small = n == SHAPES[0][0]
    dt = dtype_of(prec)
    plan = g.Plan(n, p, fam, plan_prec(g, prec))
    X = [dev(x, dt) for x in XT[:2]] + [None]
    tol = 1e-9 if prec == "fp64" else 1e-6
    opts = g.glam_opts_default(tol=tol, max_outer=200, lambda_min_ratio=5e-2)
    if small:
        lams, thetas, _, _ = O.fit_path(d, nlambda=4, ratio=5e-2, tol=1e-10)
        res = g.glam_fit_path(plan, X, dev(Y, dt), dev(W, dt), dev(pen, torch.float64), lambdas=list(lams),
                              opts=opts)
    else:
        res = g.glam_fit_path(plan, X, dev(Y, dt), dev(W, dt), dev(pen, torch.float64), nlambda=4, opts=opts)
    assert res.status == g.GLAM_OK, res.message
    path = host(res.path)
    for k in range(4):
        th = O.paper_array(path[k])
        r = O.kkt_residual(d, th, res.lambdas[k], lmax)
        assert r <= (1.001 * tol if prec == "fp64" else 3e-6), (k, r)
        if small:
            F, Fref = O.objective(d, th, res.lambdas[k]), O.objective(d, thetas[k], res.lambdas[k])
            assert abs(F - Fref) <= (1e-10 if prec == "fp64" else 1e-6) * abs(Fref), (k, F, Fref)
    plan.close()
