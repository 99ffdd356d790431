"""The banded specialisation of the FP64 gradient passes (glam_opts.exploit_bands; cubic B-spline
bases have 4 consecutive nonzeros per row, so each banded mode product sums 4 terms per output of
H and a short run of rows per output of G).  Not the paper's general method (dense designs), so it
is opt-in; the sums skip only exact zeros, so the fits are those of the dense passes up to the
summation order.

* the 20 x 20 x 20 Gaussian path with banded passes reaches the stored oracle path (FP64 and FP32
  plans): the oracle's KKT residual and objective at every lambda;
* a masked Poisson problem with spline bases (d = 3 and d = 2): banded and dense passes give the
  same objectives (1e-12 FP64) and the oracle's KKT conditions hold;
* designs that are not banded (normal rows), and plans with c > 1 components, are refused.
"""
import os

import numpy as np
import pytest

import gen
import oracle as O
from gpu_helpers import dev, dtype_of, gpu_or_skip, host, plan_prec

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_banded_gauss20_path_matches_oracle(prec):
    torch, g = gpu_or_skip()
    pr = gen.make_workload(0)
    gold = np.load(os.path.join(GOLDEN, "gauss20_path.npz"))
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    dt = dtype_of(prec)
    plan = g.Plan(pr.n, pr.p, pr.family, plan_prec(g, prec))
    tol = 1e-9 if prec == "fp64" else 1e-6
    res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                          dev(pr.pen_w, torch.float64), nlambda=10,
                          opts=g.glam_opts_default(tol=tol, lambda_min_ratio=1e-3, exploit_bands=1))
    assert res.status == g.GLAM_OK, res.message
    lmax = float(gold["lmax"])
    path = host(res.path)
    for k in range(10):
        th = O.paper_array(path[k])
        r = O.kkt_residual(d, th, res.lambdas[k], lmax)
        assert r <= (1e-9 if prec == "fp64" else 3e-6), (k, r)
        F, Fref = O.objective(d, th, res.lambdas[k]), float(gold["objective"][k])
        assert abs(F - Fref) <= (1e-10 if prec == "fp64" else 1e-6) * abs(Fref), (k, F, Fref)
    plan.close()


@pytest.mark.parametrize("n,p", [((41, 37, 23), (9, 8, 7)), ((45, 38), (8, 9))])
def test_banded_and_dense_passes_give_the_same_path(n, p):
    torch, g = gpu_or_skip()
    if len(n) == 3:
        pr = gen.random_problem(61, n, p, gen.POISSON, mask_frac=0.1, basis="spline", pen_w="random")
        XT, Y, W, pen = pr.XT, pr.Y, pr.W, pr.pen_w
    else:  # d = 2: spline bases in modes 1 and 2, X_3 = [1]
        rng = np.random.default_rng(61)
        XT = [gen.cubic_bspline_basis(n[0], p[0]).T.copy(), gen.cubic_bspline_basis(n[1], p[1]).T.copy(),
              np.ones((1, 1))]
        eta = 1.2 * np.tanh(O.predict_c(XT, rng.standard_normal((1, p[1], p[0]))))
        Y = rng.poisson(np.exp(eta)).astype(np.float64)
        W = np.ones_like(Y)
        W.reshape(-1)[rng.choice(W.size, W.size // 10, replace=False)] = 0.0
        pen = rng.uniform(0.5, 1.5, (1, p[1], p[0]))
    d = O.GlamData.from_c(gen.POISSON, XT, Y, W, pen)
    lmax = O.lambda_max(d)
    dt = torch.float64
    X = [dev(x, dt) for x in XT[:2]] + [dev(XT[2], dt) if len(n) == 3 else None]
    out = []
    for bands in (0, 1):
        plan = g.Plan(n, p, gen.POISSON, g.GLAM_FP64)
        res = g.glam_fit_path(plan, X, dev(Y, dt), dev(W, dt), dev(pen, dt), nlambda=5,
                              opts=g.glam_opts_default(tol=1e-9, lambda_min_ratio=5e-2, exploit_bands=bands,
                                                       max_outer=200))
        assert res.status == g.GLAM_OK, res.message
        out.append(res)
        plan.close()
    for k in range(5):
        Fd, Fb = out[0].stats[k]["objective"], out[1].stats[k]["objective"]
        assert abs(Fd - Fb) <= 1e-12 * abs(Fd), (k, Fd, Fb)
        th = O.paper_array(host(out[1].path)[k])
        assert O.kkt_residual(d, th, out[1].lambdas[k], lmax) <= 1.001e-9


def test_non_banded_designs_and_components_are_refused():
    torch, g = gpu_or_skip()
    pr = gen.random_problem(62, (15, 13, 9), (6, 5, 5), gen.GAUSSIAN, basis="normal")  # p_j > 4: not banded
    dt = torch.float64
    plan = g.Plan(pr.n, pr.p, pr.family, g.GLAM_FP64)
    with pytest.raises(g.GlamError) as ei:
        g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt), dev(pr.pen_w, dt),
                        nlambda=2, opts=g.glam_opts_default(exploit_bands=1))
    assert "exploit_bands" in str(ei.value)
    plan.close()
    ps = ((4, 4, 4), (4, 4, 4))
    pc = g.PlanC(pr.n, ps, pr.family, g.GLAM_FP64)
    sp = gen.random_problem(63, (15, 13, 9), (4, 4, 4), gen.GAUSSIAN, basis="spline")
    X = [[dev(x, dt) for x in sp.XT], [dev(x, dt) for x in sp.XT]]
    with pytest.raises(g.GlamError):
        g.glam_fit_path(pc, X, dev(sp.Y, dt), dev(sp.W, dt), dev(np.ones(128), dt), nlambda=2,
                        opts=g.glam_opts_default(exploit_bands=1))
    pc.close()
