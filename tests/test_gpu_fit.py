"""Parity of the GPU lambda path (glam_fit_path) with the oracle.

The target of every lambda is the minimiser of Eq. (five) (the lasso KKT conditions), which the
oracle reaches by running Algorithm 1 in FP64 to KKT 1e-10.  Parity is assessed on the solution's
objective, its linear predictor, the KKT residual evaluated by the oracle, and the active set
(exactly, except degenerate coordinates: zero in the oracle with |g_m| within 1e-6 lambda_max of
the threshold, or |theta_m| <= 1e-9 max|theta|).  The iteration trajectory is not compared.
"""
import os

import numpy as np
import pytest

import gen
import oracle as O
from gpu_helpers import (BAR, assert_within, cell_scales, chain_G, chain_H, dev, dtype_of, f32_rounded,
                         gpu_or_skip, host, plan_prec, rel_err)

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _active_sets_agree(d, th_gpu, th_ref, lam, lmax, r_tot):
    """Active sets agree except on degenerate coordinates.  Two points whose KKT residuals sum to
    r_tot (scaled by lambda_max) can differ by at most r_tot lambda_max / mu_A in theta (mu_A: the
    smallest eigenvalue of the Hessian on the active set, from the explicit design), so an active
    coordinate smaller than that bound, or an inactive one whose subgradient slack is below
    r_tot lambda_max, may legitimately flip."""
    g = O.gradient(d, th_ref)
    thr = lam * d.pen_w
    act = th_ref != 0
    Phi = O.kron_design(d.Xs)
    eta = O.H(d.Xs, th_ref)
    w = O.vec(O.irls_weight(d.family, eta, d.a))
    ia = np.flatnonzero(O.vec(act))
    bound = 0.0
    if ia.size:
        Hs = Phi[:, ia].T @ (w[:, None] * Phi[:, ia]) / d.n
        mu = max(np.linalg.eigvalsh(Hs).min(), 1e-300)
        bound = 10.0 * r_tot * lmax / mu
    # values at rounding level are not active in any meaningful sense (at lambda = lambda_max the
    # soft threshold of |z| equal to the threshold up to one rounding can leave ~1e-20)
    bound = max(bound, 1e-12 * max(1.0, float(np.abs(th_ref).max())))
    degenerate = (~act & (np.abs(np.abs(g) - thr) <= 10.0 * r_tot * lmax)) | (act & (np.abs(th_ref) <= bound))
    ok = ~degenerate
    return np.array_equal((th_gpu != 0)[ok], (th_ref != 0)[ok]), int(degenerate.sum())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gauss20_path_matches_oracle(prec):
    torch, g = gpu_or_skip()
    pr = gen.make_workload(0)
    gold = np.load(os.path.join(GOLDEN, "gauss20_path.npz"))
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    dt = dtype_of(prec)
    plan = g.Plan(pr.n, pr.p, pr.family, plan_prec(g, prec))
    tol = 1e-9 if prec == "fp64" else 1e-6
    res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                          dev(pr.pen_w, torch.float64), nlambda=10,
                          opts=g.glam_opts_default(tol=tol, lambda_min_ratio=1e-3))
    assert res.status == g.GLAM_OK, res.message
    lmax = float(gold["lmax"])
    np.testing.assert_allclose(res.lambdas, gold["lambdas"], rtol=1e-12 if prec == "fp64" else 1e-6)
    path = host(res.path)
    for k in range(10):
        th = O.paper_array(path[k])
        ref = O.paper_array(gold["thetas"][k])
        lam = res.lambdas[k]
        # KKT of the returned solution, evaluated by the oracle on the FP64 data
        r = O.kkt_residual(d, th, lam, lmax)
        assert r <= (1e-9 if prec == "fp64" else 3e-6), (k, r)
        F, Fref = O.objective(d, th, lam), float(gold["objective"][k])
        assert abs(F - Fref) <= (1e-10 if prec == "fp64" else 1e-6) * abs(Fref), (k, F, Fref)
        assert rel_err(O.H(d.Xs, th), O.H(d.Xs, ref)) <= (1e-6 if prec == "fp64" else 1e-4)
        same, ndeg = _active_sets_agree(d, th, ref, lam, lmax, r + float(gold["kkt"][k]))
        assert same, (k, ndeg)
        assert res.stats[k]["kkt"] <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON])
def test_small_masked_path_matches_oracle(prec, fam):
    torch, g = gpu_or_skip()
    n, p = (13, 11, 9), (5, 4, 4)
    pr = gen.random_problem(11, n, p, fam, mask_frac=0.15, basis="normal", pen_w="rand")
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    lams, thetas, stats, lmax = O.fit_path(d, nlambda=6, ratio=1e-2, tol=1e-10)
    dt = dtype_of(prec)
    plan = g.Plan(n, p, fam, plan_prec(g, prec))
    tol = 1e-9 if prec == "fp64" else 1e-6
    res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                          dev(pr.pen_w, torch.float64), lambdas=list(lams),
                          opts=g.glam_opts_default(tol=tol))
    assert res.status == g.GLAM_OK, res.message
    path = host(res.path)
    for k in range(len(lams)):
        th = O.paper_array(path[k])
        r = O.kkt_residual(d, th, lams[k], lmax)
        assert r <= (1e-9 if prec == "fp64" else 3e-6)
        F, Fref = O.objective(d, th, lams[k]), O.objective(d, thetas[k], lams[k])
        assert abs(F - Fref) <= (1e-10 if prec == "fp64" else 1e-6) * abs(Fref)
        np.testing.assert_allclose(th, thetas[k], atol=(1e-7 if prec == "fp64" else 1e-4) * max(1, np.abs(thetas[k]).max()))
        same, ndeg = _active_sets_agree(d, th, thetas[k], lams[k], lmax, r + stats[k].kkt)
        assert same, (k, ndeg, np.flatnonzero(O.vec(th) != 0), np.flatnonzero(O.vec(thetas[k]) != 0))


def test_lambda_max_gives_exact_zero_and_gaussian_needs_no_line_search():
    torch, g = gpu_or_skip()
    pr = gen.random_problem(12, (20, 17, 15), (6, 5, 5), gen.GAUSSIAN, mask_frac=0.1, basis="normal")
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    plan = g.Plan(pr.n, pr.p, pr.family, g.GLAM_FP64)
    res = g.glam_fit_path(plan, [dev(x, torch.float64) for x in pr.XT], dev(pr.Y, torch.float64),
                          dev(pr.W, torch.float64), dev(pr.pen_w, torch.float64), nlambda=5,
                          opts=g.glam_opts_default(lambda_min_ratio=1e-2))
    assert res.status == g.GLAM_OK
    assert abs(res.lambdas[0] - O.lambda_max(d)) <= 1e-12 * res.lambdas[0]
    assert torch.count_nonzero(res.path[0]).item() == 0
    assert torch.count_nonzero(res.path[1]).item() > 0
    assert all(s["armijo_backtracks"] == 0 for s in res.stats)


def test_iteration_cap_returns_partial_path():
    torch, g = gpu_or_skip()
    pr = gen.random_problem(13, (20, 17, 15), (6, 5, 5), gen.POISSON, basis="normal")
    plan = g.Plan(pr.n, pr.p, pr.family, g.GLAM_FP32)
    dt = torch.float32
    res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                          dev(pr.pen_w, torch.float64), nlambda=5,
                          opts=g.glam_opts_default(max_outer=1, max_inner=2, lambda_min_ratio=1e-2))
    assert res.status == g.GLAM_ENOCONV
    assert 1 <= res.nfit < 5
    assert res.stats[res.nfit]["status"] == g.GLAM_ENOCONV


def test_nonfinite_input_is_reported():
    torch, g = gpu_or_skip()
    pr = gen.random_problem(14, (10, 9, 8), (4, 4, 4), gen.GAUSSIAN, basis="normal")
    Y = pr.Y.copy()
    Y[3, 2, 1] = np.nan
    plan = g.Plan(pr.n, pr.p, pr.family, g.GLAM_FP64)
    with pytest.raises(g.GlamError) as e:
        g.glam_fit_path(plan, [dev(x, torch.float64) for x in pr.XT], dev(Y, torch.float64),
                        dev(pr.W, torch.float64), dev(pr.pen_w, torch.float64), nlambda=3)
    assert e.value.status == g.GLAM_ENONFINITE


def test_resume_from_a_warm_start():
    """A path split in two, the second half started from the first half's last solution
    (Theta0), reaches the same solutions as the uninterrupted path."""
    torch, g = gpu_or_skip()
    pr = gen.random_problem(15, (16, 14, 12), (5, 5, 4), gen.POISSON, mask_frac=0.1, basis="normal")
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    plan = g.Plan(pr.n, pr.p, pr.family, g.GLAM_FP64)
    X = [dev(x, torch.float64) for x in pr.XT]
    Y, W, pw = dev(pr.Y, torch.float64), dev(pr.W, torch.float64), dev(pr.pen_w, torch.float64)
    o = g.glam_opts_default(tol=1e-10, lambda_min_ratio=1e-2)
    full = g.glam_fit_path(plan, X, Y, W, pw, nlambda=6, opts=o)
    a = g.glam_fit_path(plan, X, Y, W, pw, lambdas=full.lambdas[:3], opts=o)
    b = g.glam_fit_path(plan, X, Y, W, pw, lambdas=full.lambdas[3:], opts=o, Theta0=a.path[2].contiguous())
    lmax = O.lambda_max(d)
    for k in range(3):
        th_full = O.paper_array(host(full.path[3 + k]))
        th_res = O.paper_array(host(b.path[k]))
        lam = full.lambdas[3 + k]
        assert abs(O.objective(d, th_full, lam) - O.objective(d, th_res, lam)) <= 1e-11 * abs(O.objective(d, th_full, lam))
        assert O.kkt_residual(d, th_res, lam, lmax) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_unfused_shape_path_matches_oracle(prec):
    """p2 = 33 exceeds the fused slab kernel's limit: the inner iteration runs the unfused chain
    of mode products and the separate prox kernel; the solutions must still meet the oracle."""
    torch, g = gpu_or_skip()
    n, p = (7, 36, 5), (3, 33, 2)
    pr = gen.random_problem(16, n, p, gen.POISSON, mask_frac=0.1, basis="normal")
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    lams, thetas, stats, lmax = O.fit_path(d, nlambda=4, ratio=5e-2, tol=1e-10)
    dt = dtype_of(prec)
    plan = g.Plan(n, p, pr.family, plan_prec(g, prec))
    res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                          dev(pr.pen_w, torch.float64), lambdas=list(lams),
                          opts=g.glam_opts_default(tol=1e-9 if prec == "fp64" else 1e-6))
    assert res.status == g.GLAM_OK, res.message
    for k in range(len(lams)):
        th = O.paper_array(host(res.path[k]))
        assert O.kkt_residual(d, th, lams[k], lmax) <= (1e-9 if prec == "fp64" else 3e-6)
        F, Fref = O.objective(d, th, lams[k]), O.objective(d, thetas[k], lams[k])
        assert abs(F - Fref) <= (1e-10 if prec == "fp64" else 1e-6) * abs(Fref)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", [gen.BINOMIAL, gen.GAMMA])
def test_binomial_and_gamma_paths_match_oracle(prec, fam):
    """The binomial (logit) and Gamma (log link) families: KKT of every returned solution,
    evaluated by the oracle, and the oracle's objectives.  The Gamma log link is not canonical:
    its Fisher weight understates the curvature where y > mu, the line search backtracks, and
    the FP64 oracle meets KKT 1e-8 (not 1e-10) in its iteration budget, so the bars follow."""
    torch, g = gpu_or_skip()
    n, p = (13, 11, 9), (5, 4, 4)
    pr = gen.random_problem(11, n, p, fam, mask_frac=0.15, basis="normal", pen_w="rand")
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    otol = 1e-8 if fam == gen.GAMMA else 1e-10
    lams, thetas, stats, lmax = O.fit_path(d, nlambda=4, ratio=1e-2, tol=otol, max_outer=400)
    # (near its optimum the oracle's Armijo test compares objective values at rounding level and
    # may stop a little short of 1e-8 for the Gamma family; the GPU compares per-cell changes)
    assert all(st.kkt <= (1e-6 if fam == gen.GAMMA else otol) for st in stats)
    dt = dtype_of(prec)
    plan = g.Plan(n, p, fam, plan_prec(g, prec))
    tol = (1e-8 if fam == gen.GAMMA else 1e-9) if prec == "fp64" else 1e-6
    res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                          dev(pr.pen_w, torch.float64), lambdas=list(lams),
                          opts=g.glam_opts_default(tol=tol, max_outer=200))
    assert res.status == g.GLAM_OK, res.message
    path = host(res.path)
    for k in range(len(lams)):
        th = O.paper_array(path[k])
        r = O.kkt_residual(d, th, lams[k], lmax)
        assert r <= (3 * tol if prec == "fp64" else 3e-6), (k, r)
        F, Fref = O.objective(d, th, lams[k]), O.objective(d, thetas[k], lams[k])
        if fam == gen.GAMMA:  # at least as good as the oracle's point, and close to it
            assert F <= Fref + 1e-10 * abs(Fref), (k, F, Fref)
            assert Fref - F <= 1e-6 * abs(Fref), (k, F, Fref)
        else:
            assert abs(F - Fref) <= (1e-9 if prec == "fp64" else 1e-6) * abs(Fref), (k, F, Fref)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON])
def test_scad_path_matches_oracle(prec, fam):
    """SCAD by the multistep adaptive lasso (penalty = GLAM_PENALTY_SCAD, 3 steps per lambda)
    against the oracle's MSA path: the solutions agree, and each meets the KKT conditions of its
    last weighted-lasso step with the weights the oracle derives from its own previous step (the
    two sides' previous steps agree to their KKT tolerance, and the SCAD weights are continuous
    in theta)."""
    torch, g = gpu_or_skip()
    n, p = (13, 11, 9), (5, 4, 4)
    pr = gen.random_problem(71, n, p, fam, mask_frac=0.1, basis="normal")
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    lmax = O.lambda_max(d)
    lams = list(lmax * np.array([1.0, 0.4, 0.15, 0.05]))
    thetas, stats, weights, _ = O.scad_path(d, lams, steps=3, tol=1e-11)
    dt = dtype_of(prec)
    plan = g.Plan(n, p, fam, plan_prec(g, prec))
    tol = 1e-10 if prec == "fp64" else 1e-7
    res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                          dev(pr.pen_w, torch.float64), lambdas=lams,
                          opts=g.glam_opts_default(tol=tol, penalty=g.GLAM_PENALTY_SCAD, steps=3))
    assert res.status == g.GLAM_OK, res.message
    path = host(res.path)
    for k in range(len(lams)):
        th = O.paper_array(path[k])
        scale = max(1.0, float(np.abs(thetas[k]).max()))
        np.testing.assert_allclose(th, thetas[k], atol=(1e-7 if prec == "fp64" else 1e-4) * scale)
        dk = O.GlamData(d.family, d.Xs, d.Y, d.a, weights[k])
        assert O.kkt_residual(dk, th, lams[k], lmax) <= (1e-7 if prec == "fp64" else 1e-4), k


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON])
@pytest.mark.parametrize("pen", ["enet", "ridge"])
def test_enet_and_ridge_paths_match_oracle(prec, fam, pen):
    """The elastic net J = sum w (|theta| + alpha theta^2) and the ridge penalty J = sum w theta^2
    (Sec. 6.3 prox forms) against the oracle: the KKT conditions of every returned solution (the
    distance of -grad f to lambda dJ, the definition of the solution), and for the Gaussian family
    the oracle's own path (objectives and solutions; both problems are strictly convex).  (The
    FP64 oracle's Armijo test compares objective values and, for Poisson ridge fits near
    lambda_max, stops at KKT ~1e-8; there the KKT conditions alone decide.)"""
    torch, g = gpu_or_skip()
    n, p = (13, 11, 9), (5, 4, 4)
    pr = gen.random_problem(91, n, p, fam, mask_frac=0.1, basis="normal", pen_w="rand")
    l1, l2, code = (1.0, 0.6, g.GLAM_PENALTY_ENET) if pen == "enet" else (0.0, 1.0, g.GLAM_PENALTY_RIDGE)
    d0 = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    d = O.GlamData(d0.family, d0.Xs, d0.Y, d0.a, d0.pen_w, l1, l2)
    lmax = O.lambda_max(d)
    lams = O.lambda_sequence(lmax, 4, 1e-2)
    if fam == gen.GAUSSIAN:
        _, thetas, stats, _ = O.fit_path(d, nlambda=4, ratio=1e-2, tol=1e-10)
        assert all(st.converged for st in stats)
    dt = dtype_of(prec)
    plan = g.Plan(n, p, fam, plan_prec(g, prec))
    tol = 1e-9 if prec == "fp64" else 1e-6
    res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                          dev(pr.pen_w, torch.float64), nlambda=4,
                          opts=g.glam_opts_default(tol=tol, lambda_min_ratio=1e-2, penalty=code,
                                                   enet_alpha=l2 if pen == "enet" else 0.0))
    assert res.status == g.GLAM_OK, res.message
    np.testing.assert_allclose(res.lambdas, lams, rtol=1e-10 if prec == "fp64" else 1e-6)
    path = host(res.path)
    for k in range(4):
        th = O.paper_array(path[k])
        r = O.kkt_residual(d, th, lams[k], lmax)
        assert r <= (1e-9 if prec == "fp64" else 3e-6), (k, r)
        assert res.stats[k]["kkt"] <= tol
        if fam == gen.GAUSSIAN:
            F, Fref = O.objective(d, th, lams[k]), O.objective(d, thetas[k], lams[k])
            assert abs(F - Fref) <= (1e-10 if prec == "fp64" else 1e-6) * abs(Fref), (k, F, Fref)
            scale = max(1.0, float(np.abs(thetas[k]).max()))
            np.testing.assert_allclose(th, thetas[k], atol=(1e-7 if prec == "fp64" else 1e-4) * scale)
    if pen == "ridge":  # no coefficient is set to zero below lambda_max
        assert np.count_nonzero(path[-1]) == path[-1].size


# ------------------------------------------------------------------------------------------
# FP32 plans on the shapes whose inner-loop product runs on the tensor cores (n1 <= 128 or a
# multiple of 32, n2 a multiple of 16, p1, p2 <= 32): the configuration the benchmark times.
# ------------------------------------------------------------------------------------------

def _cast32(pr):
    """The problem as an FP32 plan sees it: designs and data rounded to binary32 (the oracle then
    measures the solver, not the rounding of its inputs)."""
    pr.XT = [f32_rounded(x) for x in pr.XT]
    pr.Y, pr.W = f32_rounded(pr.Y), f32_rounded(pr.W)
    return pr


@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON])
@pytest.mark.parametrize("n,p", [((64, 32, 7), (9, 17, 4)), ((64, 24, 7), (9, 17, 4)), ((96, 48, 5), (30, 25, 3))])
def test_fp32_tensor_core_shape_path_matches_oracle(n, p, fam):
    """Masked lambda paths with GLAM_FP32 plans on tensor-core shapes: every returned solution
    against the oracle's path (objective, solution, active set) and the oracle's KKT residual."""
    torch, g = gpu_or_skip()
    pr = _cast32(gen.random_problem(61, n, p, fam, mask_frac=0.15, basis="normal", pen_w="rand"))
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    lams, thetas, stats, lmax = O.fit_path(d, nlambda=6, ratio=1e-2, tol=1e-10)
    dt = torch.float32
    plan = g.Plan(n, p, fam, g.GLAM_FP32)
    res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                          dev(pr.pen_w, torch.float64), lambdas=list(lams), opts=g.glam_opts_default(tol=1e-6))
    assert res.status == g.GLAM_OK, res.message
    path = host(res.path)
    for k in range(len(lams)):
        th = O.paper_array(path[k])
        r = O.kkt_residual(d, th, lams[k], lmax)
        assert r <= 1.001e-6, (k, r)
        F, Fref = O.objective(d, th, lams[k]), O.objective(d, thetas[k], lams[k])
        assert abs(F - Fref) <= 1e-6 * abs(Fref), (k, F, Fref)
        np.testing.assert_allclose(th, thetas[k], atol=1e-4 * max(1, np.abs(thetas[k]).max()))
        same, ndeg = _active_sets_agree(d, th, thetas[k], lams[k], lmax, r + stats[k].kkt)
        assert same, (k, ndeg)


def _slack_degenerate(d, th, lam, lmax, r_tot):
    """Coordinates whose zero/nonzero status two points within KKT r_tot of the solution may
    legitimately disagree on, judged from the oracle gradient alone (for problems too large for
    the explicit design): inactive ones whose subgradient slack is below 10 r_tot lambda_max and
    active ones smaller than 1e-3 of the largest coefficient."""
    gr = O.gradient(d, th)
    act = th != 0
    small = np.abs(th) <= 1e-3 * max(np.abs(th).max(), 1e-300)
    return (~act & (np.abs(np.abs(gr) - lam * d.pen_w) <= 10.0 * r_tot * lmax)) | (act & small)


def test_fp32_and_fp64_plans_on_128x128x160_meet_the_oracle_kkt():
    """A 128 x 128 x 160 Gaussian problem (p = (20, 20, 12)): the FP32 plan (tensor-core inner
    product) and the FP64 plan (FP64 SIMT products) each reach the oracle's KKT conditions at every
    lambda; their objectives agree, and so do their active sets outside degenerate coordinates."""
    torch, g = gpu_or_skip()
    n, p = (128, 128, 160), (20, 20, 12)
    pr = _cast32(gen.random_problem(62, n, p, gen.GAUSSIAN, mask_frac=0.1, basis="normal"))
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    lmax = O.lambda_max(d)
    lams = list(O.lambda_sequence(lmax, 6, 1e-2))
    out = {}
    for prec, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        plan = g.Plan(n, p, gen.GAUSSIAN, plan_prec(g, prec))
        res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                              dev(pr.pen_w, torch.float64), lambdas=lams, opts=g.glam_opts_default(tol=1e-7))
        assert res.status == g.GLAM_OK, (prec, res.message)
        out[prec] = host(res.path)
        plan.close()
    for k in range(len(lams)):
        th32, th64 = O.paper_array(out["fp32"][k]), O.paper_array(out["fp64"][k])
        r32 = O.kkt_residual(d, th32, lams[k], lmax)
        r64 = O.kkt_residual(d, th64, lams[k], lmax)
        assert r32 <= 1.001e-7 and r64 <= 1.001e-7, (k, r32, r64)
        F32, F64 = O.objective(d, th32, lams[k]), O.objective(d, th64, lams[k])
        assert abs(F32 - F64) <= 1e-9 * abs(F64), (k, F32, F64)
        deg = _slack_degenerate(d, th64, lams[k], lmax, r32 + r64)
        assert np.array_equal((th32 != 0)[~deg], (th64 != 0)[~deg]), (k, int(deg.sum()))


def test_full_workload_fp32_path_meets_the_oracle_kkt():
    """The benchmark's workload, 128 x 128 x 600 Gaussian with cubic B-spline bases p = (20, 20,
    60), 50 lambdas to KKT 1e-6 with a GLAM_FP32 plan: the oracle's KKT residual of the returned
    solution at the first, middle and last lambda, and the objective decreasing along the path."""
    torch, g = gpu_or_skip()
    pr = _cast32(gen.make_workload(1))
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    dt = torch.float32
    plan = g.Plan(pr.n, pr.p, pr.family, g.GLAM_FP32)
    res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                          dev(pr.pen_w, torch.float64), nlambda=pr.nlambda,
                          opts=g.glam_opts_default(tol=1e-6, lambda_min_ratio=1e-3))
    assert res.status == g.GLAM_OK, res.message
    lmax = O.lambda_max(d)
    assert abs(res.lambdas[0] - lmax) <= 1e-10 * lmax
    for k in (0, pr.nlambda // 2 - 1, pr.nlambda - 1):
        th = O.paper_array(host(res.path[k]))
        r = O.kkt_residual(d, th, res.lambdas[k], lmax)
        assert r <= 1.001e-6, (k, r)
        assert abs(O.objective(d, th, res.lambdas[k]) - res.stats[k]["objective"]) <= 1e-9 * abs(res.stats[k]["objective"])
    objs = [s["objective"] for s in res.stats]
    assert all(b < a for a, b in zip(objs, objs[1:]))


def test_masked_poisson_workload_path_meets_the_oracle_kkt():
    """The 96 x 96 x 365 Poisson workload (log-rate in [-2, 4], 10% of cells masked by W = 0,
    p = (30, 30, 40)), its 30-lambda path to KKT 1e-6 with a GLAM_FP32 plan: the oracle's KKT
    residual at the first, middle and last lambda."""
    torch, g = gpu_or_skip()
    pr = _cast32(gen.make_workload(2))
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    dt = torch.float32
    plan = g.Plan(pr.n, pr.p, pr.family, g.GLAM_FP32)
    res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                          dev(pr.pen_w, torch.float64), nlambda=pr.nlambda,
                          opts=g.glam_opts_default(tol=1e-6, lambda_min_ratio=1e-3))
    assert res.status == g.GLAM_OK, res.message
    lmax = O.lambda_max(d)
    for k in (0, pr.nlambda // 2 - 1, pr.nlambda - 1):
        th = O.paper_array(host(res.path[k]))
        r = O.kkt_residual(d, th, res.lambdas[k], lmax)
        assert r <= 1.001e-6, (k, r)
        F = O.objective(d, th, res.lambdas[k])
        assert abs(F - res.stats[k]["objective"]) <= 1e-9 * abs(F)


# ------------------------------------------------------------------------------------------
# d = 2 (n3 = p3 = 1, X[2] = None: the trivial third mode of Sec. 6.4's d = 2, 3)
# ------------------------------------------------------------------------------------------

def _two_d(seed, n2d, p2d, fam, mask=0.1):
    pr = gen.random_problem(seed, n2d + (1,), p2d + (1,), fam, mask_frac=mask, basis="normal", pen_w="rand")
    pr.XT[2] = np.ones((1, 1))
    return pr


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON])
def test_two_dimensional_gradient_and_path_match_oracle(prec, fam):
    torch, g = gpu_or_skip()
    n2d, p2d = (45, 31), (7, 9)
    pr = _two_d(63, n2d, p2d, fam)
    if prec == "fp32":
        pr = _cast32(pr)
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    dt = dtype_of(prec)
    plan = g.Plan(n2d, p2d, fam, plan_prec(g, prec))
    X = [dev(pr.XT[0], dt), dev(pr.XT[1], dt), None]
    theta = 0.3 * np.random.default_rng(64).standard_normal((1, p2d[1], p2d[0]))
    grad = host(g.glam_gradient(plan, X, dev(theta, dt), dev(pr.Y, dt), dev(pr.W, dt)))
    th = O.paper_array(theta)
    su, _, _ = cell_scales(fam, O.H(d.Xs, th), chain_H(d.Xs, th), d.Y, d.a)
    assert_within(grad, O.c_array(O.gradient(d, th)), O.c_array(chain_G(d.Xs, su)) / d.n, BAR[prec],
                  what="grad (d = 2)")
    lams, thetas, stats, lmax = O.fit_path(d, nlambda=5, ratio=1e-2, tol=1e-10)
    tol = 1e-9 if prec == "fp64" else 1e-6
    res = g.glam_fit_path(plan, X, dev(pr.Y, dt), dev(pr.W, dt), dev(pr.pen_w, torch.float64),
                          lambdas=list(lams), opts=g.glam_opts_default(tol=tol))
    assert res.status == g.GLAM_OK, res.message
    for k in range(len(lams)):
        thk = O.paper_array(host(res.path[k]))
        r = O.kkt_residual(d, thk, lams[k], lmax)
        assert r <= 1.001 * tol, (k, r)
        F, Fref = O.objective(d, thk, lams[k]), O.objective(d, thetas[k], lams[k])
        assert abs(F - Fref) <= (1e-10 if prec == "fp64" else 1e-6) * abs(Fref)
        same, ndeg = _active_sets_agree(d, thk, thetas[k], lams[k], lmax, r + stats[k].kkt)
        assert same, (k, ndeg)
