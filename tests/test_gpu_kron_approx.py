"""The geometric-mean tensor approximation of the weights (iwls kron1 / kron2, Sec. 6.2 and the
iwls option of Sec. 6.4) and the inner step-size option nu < 1 (Sec. 6.4), against the oracle.

* glam_kron_weights gives the oracle's factors (masked cells excluded) to FP64 rounding, for a
  ragged shape with several slabs and a d = 2 shape;
* a fit with either approximation reaches the exact-weight solutions (Sec. 5: any positive weights
  keep the fixed point): the oracle's KKT residual of every returned solution and the objectives
  of the exact-weight path;
* nu = 0.5 and nu = 0 reach the same solutions; where the first step 1 / (nu L_hat) (or 1) is too
  long the solve restarts with a halved step and the restarts are reported.
"""
import numpy as np
import pytest

import gen
import oracle as O
from gpu_helpers import dev, dtype_of, gpu_or_skip, host, plan_prec

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [(37, 29, 13), (40, 33, 1)])
@pytest.mark.parametrize("scaled", [False, True])
def test_kron_weights_match_oracle(n, scaled):
    torch, g = gpu_or_skip()
    rng = np.random.default_rng(31)
    V = rng.uniform(0.05, 4.0, (n[2], n[1], n[0]))  # C-order (n3, n2, n1)
    V[rng.random(V.shape) < 0.1] = 0.0              # masked cells
    V[:, 3, :] = 0.0                                # a slice of mode 2 with no positive cell
    p = (3, 3, 1 if n[2] == 1 else 3)
    plan = g.Plan(n, p, gen.POISSON, g.GLAM_FP64)
    got = g.glam_kron_weights(plan, dev(V, torch.float64), scaled=scaled)
    ref = O.geometric_mean_weights(O.paper_array(V), scaled=scaled)
    for j in range(3):
        a, b = host(got[j]), ref[j]
        assert a.shape == b.shape
        assert np.allclose(a, b, rtol=1e-12, atol=0.0), (j, np.max(np.abs(a - b) / b))
    assert host(got[1])[3] == 1.0
    again = g.glam_kron_weights(plan, dev(V, torch.float64), scaled=scaled)
    for j in range(3):  # fixed summation order: the same bits
        assert np.array_equal(host(got[j]), host(again[j]))
    plan.close()


def _fit(g, torch, pr, prec, nlambda, **opt):
    dt = dtype_of(prec)
    plan = g.Plan(pr.n, pr.p, pr.family, plan_prec(g, prec))
    res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                          dev(pr.pen_w, torch.float64), nlambda=nlambda,
                          opts=g.glam_opts_default(**opt))
    plan.close()
    return res


def _cast(prec):
    if prec == "fp64":
        return lambda a: np.asarray(a, np.float64)
    return lambda a: np.asarray(a, np.float32).astype(np.float64)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", [gen.POISSON, gen.BINOMIAL])
def test_kron_approximations_reach_exact_solutions(prec, fam):
    torch, g = gpu_or_skip()
    pr = gen.random_problem(33, (37, 29, 13), (9, 7, 6), fam, mask_frac=0.1, basis="normal",
                            pen_w="random")
    c = _cast(prec)
    pr.XT = [c(x) for x in pr.XT]
    pr.Y, pr.W = c(pr.Y), c(pr.W)
    d = O.GlamData.from_c(fam, pr.XT, pr.Y, pr.W, pr.pen_w)
    lmax = O.lambda_max(d)
    tol = 1e-8 if prec == "fp64" else 1e-6
    base = dict(tol=tol, lambda_min_ratio=5e-2, max_outer=300)
    ref = _fit(g, torch, pr, prec, 4, **base)
    assert ref.status == g.GLAM_OK, ref.message
    for iwls in (g.GLAM_IWLS_KRON1, g.GLAM_IWLS_KRON2):
        res = _fit(g, torch, pr, prec, 4, iwls=iwls, **base)
        assert res.status == g.GLAM_OK, (iwls, res.message)
        assert np.allclose(res.lambdas, ref.lambdas, rtol=1e-12)
        path = host(res.path)
        for k in range(4):
            th = O.paper_array(path[k])
            r = O.kkt_residual(d, th, res.lambdas[k], lmax)
            assert r <= (2 * tol if prec == "fp64" else 3e-6), (iwls, k, r)
            F, Fe = O.objective(d, th, res.lambdas[k]), ref.stats[k]["objective"]
            assert abs(F - Fe) <= (1e-9 if prec == "fp64" else 1e-6) * abs(Fe), (iwls, k, F, Fe)


@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON])
def test_inner_step_option_nu_reaches_the_same_solutions(fam):
    """Designs with unit-variance rows (no 1/sqrt(n_j) scaling): L_hat is well above 1, so nu = 0
    (first step 1) and nu = 0.5 (first step 2 / L_hat) both start past 1 / L_hat."""
    torch, g = gpu_or_skip()
    pr = gen.random_problem(34, (23, 19, 11), (6, 5, 4), fam, mask_frac=0.05, basis="normal")
    pr.XT = [x * np.sqrt(x.shape[1]) for x in pr.XT]
    if fam == gen.GAUSSIAN:
        pr.Y = O.c_array(O.H([x.T for x in pr.XT], O.paper_array(0.1 * np.ones((4, 5, 6))))) + \
            0.3 * np.random.default_rng(35).standard_normal(pr.Y.shape)
    d = O.GlamData.from_c(fam, pr.XT, pr.Y, pr.W, pr.pen_w)
    lmax = O.lambda_max(d)
    rho = np.prod([O.spectral_radius_gram(X) for X in d.Xs])
    assert rho / d.n > 2.0  # L_hat > 1 (w >= 1 somewhere for these data)
    base = dict(tol=1e-9, lambda_min_ratio=5e-2, max_outer=300)
    ref = _fit(g, torch, pr, "fp64", 3, **base)
    assert ref.status == g.GLAM_OK, ref.message
    for nu in (0.5, 0.0):
        res = _fit(g, torch, pr, "fp64", 3, nu=nu, **base)
        assert res.status == g.GLAM_OK, (nu, res.message)
        path = host(res.path)
        for k in range(3):
            th = O.paper_array(path[k])
            assert O.kkt_residual(d, th, res.lambdas[k], lmax) <= 2e-9, (nu, k)
            Fe = ref.stats[k]["objective"]
            assert abs(O.objective(d, th, res.lambdas[k]) - Fe) <= 1e-11 * abs(Fe), (nu, k)
        if nu == 0.0:
            assert sum(s["inner_restarts"] for s in res.stats[:3]) >= 1
    assert all(s["inner_restarts"] == 0 for s in ref.stats[:3])


def test_nu_out_of_range_is_refused():
    torch, g = gpu_or_skip()
    pr = gen.random_problem(36, (9, 8, 7), (4, 4, 4), gen.GAUSSIAN, basis="normal")
    for nu in (-0.1, 1.5):
        with pytest.raises(g.GlamError):
            _fit(g, torch, pr, "fp64", 2, nu=nu)
