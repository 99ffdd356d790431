"""Plans of the model with c > 1 components (Sec. 2, Eq. fivenew; Eqs. eighteen/nineteen with
r = 1..c; Prop. 1 with the sum over r) against the oracle.

* glam_predict, glam_gradient and glam_loss with two components (d = 3, ragged sizes) and three
  components (d = 2), all four families, FP64 and FP32 plans, element by element against the
  absolute-value chain of each component;
* glam_fit_path with two components (Gaussian and masked Poisson, FP64 and FP32 plans) reaches
  the oracle's solutions: the oracle's KKT residual and objective at every returned lambda;
* c = 1 through glam_plan_create_components is the plain plan (the same bits);
* the entry points that take one component refuse a c > 1 plan.
"""
import numpy as np
import pytest

import gen
import oracle as O
from gpu_helpers import BAR, assert_within, cell_scales, chain_G, chain_H, dev, dtype_of, gpu_or_skip, host, \
    plan_prec

pytestmark = pytest.mark.gpu


def _problem(seed, n, ps, fam, mask=0.1):
    """c components with N(0, 1/n_j) designs, a sparse truth and the family's response; C layout
    (XTs[r][j] (p_rj, n_j), Y and W (n3, n2, n1), the flat coefficient vector)."""
    rng = np.random.default_rng(seed)
    XTs = [[rng.standard_normal((p[j], n[j])) / np.sqrt(n[j]) for j in range(3)] for p in ps]
    if n[2] == 1:  # d = 2: X_r3 = [1]
        for XT in XTs:
            XT[2] = np.ones((1, 1))
    ptot = sum(int(np.prod(p)) for p in ps)
    truth = rng.standard_normal(ptot) * (rng.random(ptot) < 0.4)
    d = O.GlamData.from_c_components(fam, XTs, np.zeros(n[::-1]), np.ones(n[::-1]), np.ones(ptot))
    eta = O.c_array(d.H(truth))
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
    pen = rng.uniform(0.5, 1.5, ptot)
    return XTs, Y, W, pen


def _cast(prec, a):
    return np.asarray(a, np.float64) if prec == "fp64" else np.asarray(a, np.float32).astype(np.float64)


def _scales(d, theta, fam):
    """|H|(|theta|) summed over the components, and the per-component |G| of the score scale."""
    eta_abs = sum(chain_H(Xr, O.unvec(np.abs(theta[o:o + k]), tuple(X.shape[1] for X in Xr)))
                  for Xr, o, k in _blocks(d))
    eta = d.H(theta)
    su, _, _ = cell_scales(d.family, eta, eta_abs, d.Y, d.a)
    gs = np.concatenate([O.vec(chain_G(Xr, su)) for Xr, _, _ in _blocks(d)]) / d.n
    return eta_abs, gs


def _blocks(d):
    o = 0
    for Xr in d.comps:
        k = int(np.prod([X.shape[1] for X in Xr]))
        yield Xr, o, k
        o += k


CASES = [((37, 29, 13), ((9, 7, 6), (5, 8, 3))),       # two components, d = 3
         ((40, 33, 1), ((7, 5, 1), (4, 9, 1), (6, 6, 1)))]  # three components, d = 2


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON, gen.BINOMIAL, gen.GAMMA])
@pytest.mark.parametrize("n,ps", CASES)
def test_components_predict_gradient_loss_match_oracle(prec, fam, n, ps):
    torch, g = gpu_or_skip()
    XTs, Y, W, pen = _problem(51, n, ps, fam)
    XTs = [[_cast(prec, x) for x in XT] for XT in XTs]
    Y, W = _cast(prec, Y), _cast(prec, W)
    d = O.GlamData.from_c_components(fam, XTs, Y, W, pen)
    dt = dtype_of(prec)
    two_d = n[2] == 1
    plan = g.PlanC(n[:2] if two_d else n, [p[:2] if two_d else p for p in ps], fam, plan_prec(g, prec))
    X = [[dev(x, dt) for x in XT[:2]] + [None if two_d else dev(XT[2], dt)] for XT in XTs]
    theta = 0.3 * np.random.default_rng(52).standard_normal(d.pshape[0])
    th = dev(theta, dt)
    eta_abs, gscale = _scales(d, theta, fam)
    eta = g.glam_predict(plan, X, th)
    assert_within(host(eta), O.c_array(d.H(theta)), O.c_array(eta_abs), BAR[prec], what="eta")
    grad, loss = g.glam_gradient(plan, X, th, dev(Y, dt), dev(W, dt), want_loss=True)
    assert_within(host(grad), O.gradient(d, theta), gscale, BAR[prec], what="grad")
    fref = O.loss(fam, d.H(theta), d.Y, d.a)
    assert abs(loss.item() - fref) <= (1e-12 if prec == "fp64" else 1e-6) * abs(fref)
    l2 = g.glam_loss(plan, X, th, dev(Y, dt), dev(W, dt))
    assert abs(l2.item() - fref) <= (1e-12 if prec == "fp64" else 1e-6) * abs(fref)
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON])
def test_components_fit_path_matches_oracle(prec, fam):
    torch, g = gpu_or_skip()
    n, ps = (23, 19, 11), ((5, 4, 4), (3, 6, 2))
    XTs, Y, W, pen = _problem(53, n, ps, fam, mask=0.1 if fam == gen.POISSON else 0.0)
    XTs = [[_cast(prec, x) for x in XT] for XT in XTs]
    Y, W = _cast(prec, Y), _cast(prec, W)
    d = O.GlamData.from_c_components(fam, XTs, Y, W, pen)
    lams, thetas, stats, lmax = O.fit_path(d, nlambda=4, ratio=5e-2, tol=1e-10)
    dt = dtype_of(prec)
    plan = g.PlanC(n, ps, fam, plan_prec(g, prec))
    X = [[dev(x, dt) for x in XT] for XT in XTs]
    tol = 1e-9 if prec == "fp64" else 1e-6
    res = g.glam_fit_path(plan, X, dev(Y, dt), dev(W, dt), dev(pen, torch.float64), lambdas=list(lams),
                          opts=g.glam_opts_default(tol=tol, max_outer=200))
    assert res.status == g.GLAM_OK, res.message
    path = host(res.path)
    for k in range(len(lams)):
        r = O.kkt_residual(d, path[k], lams[k], lmax)
        assert r <= (1.001 * tol if prec == "fp64" else 3e-6), (k, r)
        F, Fref = O.objective(d, path[k], lams[k]), O.objective(d, thetas[k], lams[k])
        assert abs(F - Fref) <= (1e-10 if prec == "fp64" else 1e-6) * abs(Fref), (k, F, Fref)
    plan.close()


def test_one_component_through_the_components_api_is_the_plain_plan():
    torch, g = gpu_or_skip()
    n, p = (21, 17, 9), (6, 5, 4)
    XTs, Y, W, pen = _problem(54, n, (p,), gen.POISSON)
    X = [dev(x, torch.float64) for x in XTs[0]]
    theta = np.random.default_rng(55).standard_normal((p[2], p[1], p[0]))
    a = g.glam_predict(g.Plan(n, p, gen.POISSON, g.GLAM_FP64), X, dev(theta, torch.float64))
    pc = g.PlanC(n, (p,), gen.POISSON, g.GLAM_FP64)
    b = g.glam_predict(pc, [X], dev(theta.reshape(-1), torch.float64))
    assert np.array_equal(host(a).reshape(-1), host(b).reshape(-1))


def test_single_component_entry_points_refuse_components_plans():
    torch, g = gpu_or_skip()
    n, ps = (15, 13, 7), ((4, 3, 3), (3, 3, 2))
    XTs, Y, W, pen = _problem(56, n, ps, gen.GAUSSIAN)
    plan = g.PlanC(n, ps, gen.GAUSSIAN, g.GLAM_FP64)
    X = [[dev(x, torch.float64) for x in XT] for XT in XTs]
    th = dev(np.zeros(plan.ncoef), torch.float64)
    with pytest.raises(g.GlamError):
        g.glam_quad_build(plan, X, th, dev(Y, torch.float64), dev(W, torch.float64))
    with pytest.raises(g.GlamError):
        g.glam_penalized_nll(plan, X, th, dev(Y, torch.float64), dev(W, torch.float64), 0.1,
                             dev(pen, torch.float64))
    with pytest.raises(g.GlamError):
        g.glam_fit_path(plan, X, dev(Y, torch.float64), dev(W, torch.float64), dev(pen, torch.float64),
                        nlambda=2, opts=g.glam_opts_default(iwls=g.GLAM_IWLS_KRON1))
    plan.close()
