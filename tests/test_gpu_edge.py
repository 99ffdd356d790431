"""Degenerate and edge shapes of the CUDA path against the oracle: single-cell and single-basis
dimensions, a one-row mode, a fully masked response (lambda_max = 0, refused), and lambda = 0
for the Gaussian family (weighted least squares by the normal equations)."""
import numpy as np
import pytest

import gen
import oracle as O
from gpu_helpers import (BAR, assert_within, cell_scales, chain_G, chain_H, dev, dtype_of, gpu_or_skip,
                         host, plan_prec)

pytestmark = pytest.mark.gpu

EDGE = [((1, 1, 1), (1, 1, 1)), ((2, 1, 3), (1, 1, 2)), ((1, 5, 1), (1, 3, 1)), ((33, 1, 2), (3, 1, 1))]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON])
@pytest.mark.parametrize("n,p", EDGE)
def test_edge_shapes_predict_gradient_loss(prec, fam, n, p):
    torch, g = gpu_or_skip()
    pr = gen.random_problem(101, n, p, fam, basis="normal")
    dt = dtype_of(prec)
    plan = g.Plan(n, p, fam, plan_prec(g, prec))
    theta = 0.3 * np.random.default_rng(102).standard_normal((p[2], p[1], p[0]))
    X = [dev(x, dt) for x in pr.XT]
    eta = g.glam_predict(plan, X, dev(theta, dt))
    grad, loss = g.glam_gradient(plan, X, dev(theta, dt), dev(pr.Y, dt), dev(pr.W, dt), want_loss=True)
    torch.cuda.synchronize()
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    th = O.paper_array(theta)
    eta_abs = chain_H(d.Xs, th)
    assert_within(host(eta), O.predict_c(pr.XT, theta), O.c_array(eta_abs), BAR[prec], what="eta")
    su, _, _ = cell_scales(fam, O.H(d.Xs, th), eta_abs, d.Y, d.a)
    assert_within(host(grad), O.c_array(O.gradient(d, th)), O.c_array(chain_G(d.Xs, su)) / d.n, BAR[prec],
                  what="grad")
    fref = O.loss(fam, O.H(d.Xs, th), d.Y, d.a)
    assert abs(loss.item() - fref) <= (1e-12 if prec == "fp64" else 1e-6) * max(1.0, abs(fref))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_edge_shape_path_meets_kkt(prec):
    torch, g = gpu_or_skip()
    n, p = (3, 2, 4), (2, 1, 2)
    pr = gen.random_problem(103, n, p, gen.GAUSSIAN, basis="normal")
    dt = dtype_of(prec)
    # the oracle sees the inputs the plan sees (rounded to FP32 for an FP32 plan)
    cast = (lambda a: np.asarray(a, np.float64)) if prec == "fp64" else (
        lambda a: np.asarray(a, np.float32).astype(np.float64))
    pr.XT, pr.Y, pr.W = [cast(x) for x in pr.XT], cast(pr.Y), cast(pr.W)
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    plan = g.Plan(n, p, pr.family, plan_prec(g, prec))
    res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                          dev(pr.pen_w, torch.float64), nlambda=3,
                          opts=g.glam_opts_default(tol=1e-8, lambda_min_ratio=1e-2))
    assert res.status == g.GLAM_OK, res.message
    lmax = O.lambda_max(d)
    for k in range(3):
        assert O.kkt_residual(d, O.paper_array(host(res.path)[k]), res.lambdas[k], lmax) <= 3e-8


def test_fully_masked_response_is_refused():
    torch, g = gpu_or_skip()
    n, p = (6, 5, 4), (3, 3, 2)
    pr = gen.random_problem(104, n, p, gen.POISSON, basis="normal")
    plan = g.Plan(n, p, gen.POISSON, g.GLAM_FP64)
    f64 = torch.float64
    with pytest.raises(g.GlamError) as e:
        g.glam_fit_path(plan, [dev(x, f64) for x in pr.XT], dev(pr.Y, f64), dev(np.zeros(pr.Y.shape), f64),
                        dev(pr.pen_w, f64), nlambda=3)
    assert e.value.status == g.GLAM_EINVAL
    assert "lambda_max" in e.value.message


def test_gaussian_lambda_zero_is_weighted_least_squares():
    torch, g = gpu_or_skip()
    n, p = (9, 7, 6), (4, 4, 3)
    pr = gen.random_problem(105, n, p, gen.GAUSSIAN, mask_frac=0.2, basis="normal")
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    plan = g.Plan(n, p, gen.GAUSSIAN, g.GLAM_FP64)
    f64 = torch.float64
    res = g.glam_fit_path(plan, [dev(x, f64) for x in pr.XT], dev(pr.Y, f64), dev(pr.W, f64),
                          dev(pr.pen_w, f64), lambdas=[0.0], opts=g.glam_opts_default(tol=1e-11))
    assert res.status == g.GLAM_OK, res.message
    Phi = O.kron_design(d.Xs)
    sw = np.sqrt(O.vec(d.a))
    ls, *_ = np.linalg.lstsq(sw[:, None] * Phi, sw * O.vec(d.Y), rcond=None)
    np.testing.assert_allclose(O.vec(O.paper_array(host(res.path)[0])), ls, rtol=1e-8, atol=1e-10)
