"""GLAM_TF32 plans: the bottleneck product G(V (.) H(y)) of Sec. 6.2 (Eq. twentysixnew) on the
tensor cores against the FP64 oracle, and lambda paths that still meet the FP64 KKT tolerance.

Tolerance, derived from the arithmetic: the tensor-core kernel rounds each of the eight operands
along the product chain (X_1 and T_a; T_b and X_2; r = V (.) eta and X_2; S and X_1) to TF32
(unit roundoff u = 2^-11, round to nearest) and accumulates in FP32.  To first order every entry
then errs by at most 8u times the same chain evaluated on absolute values,
|G|(|V| (.) |H|(|y|)); the tests allow 10u times that, plus 2e-6 of its maximum for the FP32
steps around the kernel (T_a = X_3 y, the mode-3 adjoint, the prox arithmetic).
"""
import numpy as np
import pytest

import gen
import oracle as O
from gpu_helpers import dev, gpu_or_skip, host

pytestmark = pytest.mark.gpu
U_TF32 = 2.0 ** -11

# shapes inside a tensor-core kernel's domain: the warp-level kernel (n1 % 32 == 0, n2 % 8 == 0)
# for the first four, the tcgen05 kernel (n1 <= 128, n1 % 4 == 0, n2 % 32 == 0) for the rest
TC_SHAPES = [
    ((32, 8, 3), (5, 3, 2)),          # one column group, one row block, one K step
    ((64, 24, 7), (9, 17, 4)),        # 64-column warps, p2 = 17 (three K steps), three row groups
    ((96, 40, 13), (30, 25, 6)),      # 32-column warps (n1 % 64 != 0), four K steps, uneven rows
    ((160, 16, 5), (32, 32, 3)),      # ten 16-row MMA0 tiles, p1 = p2 = 32
    ((128, 128, 160), (20, 20, 12)),  # the 128 x 128 slab, two slabs on some CTAs
    ((64, 32, 7), (9, 17, 4)),        # tcgen05: 64 lanes used, one V chunk, p2 = 17 (N 32 / 24)
    ((100, 64, 155), (7, 30, 5)),     # tcgen05: n1 = 100 (ragged last K atom), 155 slabs (two on 3 CTAs)
    ((96, 96, 31), (30, 30, 9)),      # tcgen05: the 96 x 96 slab, three V chunks, p = 30
    ((128, 96, 2), (32, 32, 1)),      # tcgen05: p1 = p2 = 32, p3 = 1, two slabs on two CTAs
]
# shapes of the tcgen05 kernel only (BF16 plans: n1 % 8 == 0 as well)
UM_SHAPES = TC_SHAPES[4:]
# shapes outside it: a TF32 plan runs the FP32 kernels there
FALLBACK_SHAPES = [((37, 29, 13), (9, 7, 6)), ((256, 64, 9), (8, 12, 5))]


def _abs_chain(Xs, V, y):
    """|G|(|V| (.) |H|(|y|)): the product with every factor replaced by its absolute value."""
    Xa = [np.abs(X) for X in Xs]
    return O.G(Xa, np.abs(V) * O.H(Xa, np.abs(y)))


def _product(g, torch, plan, X, q, x32, xp32, omega, pen):
    """y - x_next of a prox step with lambda = 0, delta = n and b = 0, i.e. G(V (.) H(y))."""
    n = float(np.prod(plan.cells_shape()))
    xn = g.glam_prox_step(plan, X, q, dev(x32, torch.float32), dev(xp32, torch.float32), omega, n,
                          0.0, pen)
    torch.cuda.synchronize()
    y = x32.astype(np.float64) + omega * (x32.astype(np.float64) - xp32.astype(np.float64))
    return y, y - host(xn)


@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON])
@pytest.mark.parametrize("n,p", TC_SHAPES + FALLBACK_SHAPES)
def test_tf32_product_parity(n, p, fam):
    torch, g = gpu_or_skip()
    pr = gen.random_problem(21, n, p, fam, mask_frac=0.1, basis="normal")
    dt = torch.float32
    X = [dev(x, dt) for x in pr.XT]
    rng = np.random.default_rng(22)
    theta_k = 0.2 * rng.standard_normal((p[2], p[1], p[0]))
    x32 = rng.standard_normal(theta_k.shape).astype(np.float32)
    xp32 = (x32 + 0.1 * rng.standard_normal(theta_k.shape)).astype(np.float32)
    pen = dev(pr.pen_w, dt)
    out = {}
    for prec in (g.GLAM_TF32, g.GLAM_FP32):
        plan = g.Plan(n, p, fam, prec)
        q = g.glam_quad_build(plan, X, dev(theta_k, dt), dev(pr.Y, dt), dev(pr.W, dt))
        q.b.zero_()
        y, got = _product(g, torch, plan, X, q, x32, xp32, 0.3, pen)
        _, again = _product(g, torch, plan, X, q, x32, xp32, 0.3, pen)
        assert np.array_equal(got, again)  # fixed summation order: the same bits on every run
        out[prec] = (got, host(q.V))
    got, Vc = out[g.GLAM_TF32]
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    Vp, yp = O.paper_array(Vc), O.paper_array(y)
    ref = O.c_array(O.G(d.Xs, Vp * O.H(d.Xs, yp)))
    scale = O.c_array(_abs_chain(d.Xs, Vp, yp))
    err = np.abs(got - ref)
    assert np.all(err <= 10 * U_TF32 * scale + 2e-6 * scale.max()), float((err / scale).max())
    # the tensor-core kernel ran on its shapes (TF32 rounding differs from the FP32 kernel),
    # and the FP32 kernels ran elsewhere (the same bits as a GLAM_FP32 plan)
    diff = np.abs(got - out[g.GLAM_FP32][0]).max() / np.abs(ref).max()
    if (n, p) in TC_SHAPES:
        assert diff > 3e-6, diff
    else:
        assert diff == 0.0, diff


@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON])
@pytest.mark.parametrize("n,p", TC_SHAPES)
def test_fp32_tensor_core_product_parity(n, p, fam):
    """GLAM_FP32 plans run the same product in the 3xTF32 form where its domain allows (each
    operand as hi + lo, both TF32, so the split leaves at most 2^-22 of it; three MMAs per product,
    the lo lo term dropped).  Bound: 32 x 2^-22 of the absolute-value chain (the split errors of
    the eight operands and the dropped terms) plus 1e-6 of its maximum for the FP32 sums."""
    torch, g = gpu_or_skip()
    pr = gen.random_problem(24, n, p, fam, mask_frac=0.1, basis="normal")
    dt = torch.float32
    X = [dev(x, dt) for x in pr.XT]
    rng = np.random.default_rng(25)
    theta_k = 0.2 * rng.standard_normal((p[2], p[1], p[0]))
    x32 = rng.standard_normal(theta_k.shape).astype(np.float32)
    xp32 = (x32 + 0.1 * rng.standard_normal(theta_k.shape)).astype(np.float32)
    plan = g.Plan(n, p, fam, g.GLAM_FP32)
    q = g.glam_quad_build(plan, X, dev(theta_k, dt), dev(pr.Y, dt), dev(pr.W, dt))
    q.b.zero_()
    y, got = _product(g, torch, plan, X, q, x32, xp32, 0.3, dev(pr.pen_w, dt))
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    Vp, yp = O.paper_array(host(q.V)), O.paper_array(y)
    ref = O.c_array(O.G(d.Xs, Vp * O.H(d.Xs, yp)))
    scale = O.c_array(_abs_chain(d.Xs, Vp, yp))
    err = np.abs(got - ref)
    assert np.all(err <= 32 * 2.0 ** -22 * scale + 1e-6 * scale.max()), float((err / scale).max())


@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON])
def test_tf32_small_path_matches_oracle(fam):
    """A masked lambda path on a tensor-core shape: the TF32 inner products only change the
    iteration count, the FP64 KKT test decides when each lambda is done."""
    torch, g = gpu_or_skip()
    from test_gpu_fit import _active_sets_agree
    n, p = (32, 16, 12), (6, 5, 4)
    pr = gen.random_problem(23, n, p, fam, mask_frac=0.15, basis="normal", pen_w="rand")
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    lams, thetas, stats, lmax = O.fit_path(d, nlambda=6, ratio=1e-2, tol=1e-10)
    dt = torch.float32
    plan = g.Plan(n, p, fam, g.GLAM_TF32)
    res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                          dev(pr.pen_w, torch.float64), lambdas=list(lams),
                          opts=g.glam_opts_default(tol=1e-6))
    assert res.status == g.GLAM_OK, res.message
    path = host(res.path)
    for k in range(len(lams)):
        th = O.paper_array(path[k])
        r = O.kkt_residual(d, th, lams[k], lmax)
        assert r <= 3e-6, (k, r)
        F, Fref = O.objective(d, th, lams[k]), O.objective(d, thetas[k], lams[k])
        assert abs(F - Fref) <= 1e-6 * abs(Fref)
        np.testing.assert_allclose(th, thetas[k], atol=1e-4 * max(1, np.abs(thetas[k]).max()))
        same, ndeg = _active_sets_agree(d, th, thetas[k], lams[k], lmax, r + stats[k].kkt)
        assert same, (k, ndeg)


def test_tf32_workload_path_agrees_with_fp32():
    """The first lambdas of the 128x128x600 Gaussian path (cubic B-spline bases, p = (20, 20, 60))
    with a TF32 plan and an FP32 plan: both meet KKT 1e-6, and their objectives agree to the
    accuracy that tolerance fixes; the oracle checks the KKT residual of the last one."""
    torch, g = gpu_or_skip()
    pr = gen.make_workload(1)
    dt = torch.float32
    X = [dev(x, dt) for x in pr.XT]
    Y, W = dev(pr.Y, dt), dev(pr.W, dt)
    pen = dev(pr.pen_w, torch.float64)
    opts = g.glam_opts_default(tol=1e-6)
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    lmax = O.lambda_max(d)
    lams = [lmax * v for v in np.geomspace(1.0, 1e-3, 50)[:6]]  # the first 6 of the 50-lambda path
    res = {}
    for prec in (g.GLAM_FP32, g.GLAM_TF32):
        plan = g.Plan(pr.n, pr.p, pr.family, prec)
        res[prec] = g.glam_fit_path(plan, X, Y, W, pen, lambdas=lams, opts=opts)
        assert res[prec].status == g.GLAM_OK, res[prec].message
        for k in range(len(lams)):
            assert res[prec].stats[k]["kkt"] <= 1e-6
    for k in range(len(lams)):
        F32 = res[g.GLAM_FP32].stats[k]["objective"]
        Ftf = res[g.GLAM_TF32].stats[k]["objective"]
        assert abs(Ftf - F32) <= 1e-6 * abs(F32), (k, Ftf, F32)
    th = O.paper_array(host(res[g.GLAM_TF32].path[5]))
    assert O.kkt_residual(d, th, lams[5], lmax) <= 3e-6



U_BF16 = 2.0 ** -8


@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON])
@pytest.mark.parametrize("n,p", [sh for sh in UM_SHAPES if sh[0][0] % 8 == 0] + [((128, 256, 3), (32, 32, 2))])
def test_bf16_product_parity(n, p, fam):
    """GLAM_BF16 plans: the product on the tcgen05 kernel with BF16 operands rounded to nearest
    (u = 2^-8) and FP32 accumulation.  The chain rounds six operands (T_b and X_2; r and X_2; P and
    X_1), so to first order every entry errs by at most 6u times the absolute-value chain; the test
    allows 8u of it plus 1e-5 of its maximum for the FP32 steps around the kernel.  The product must
    also be repeatable bit for bit and differ from the FP32 plan's (the BF16 kernel ran)."""
    torch, g = gpu_or_skip()
    pr = gen.random_problem(26, n, p, fam, mask_frac=0.1, basis="normal")
    dt = torch.float32
    X = [dev(x, dt) for x in pr.XT]
    rng = np.random.default_rng(27)
    theta_k = 0.2 * rng.standard_normal((p[2], p[1], p[0]))
    x32 = rng.standard_normal(theta_k.shape).astype(np.float32)
    xp32 = (x32 + 0.1 * rng.standard_normal(theta_k.shape)).astype(np.float32)
    pen = dev(pr.pen_w, dt)
    out = {}
    for prec in (g.GLAM_BF16, g.GLAM_FP32):
        plan = g.Plan(n, p, fam, prec)
        q = g.glam_quad_build(plan, X, dev(theta_k, dt), dev(pr.Y, dt), dev(pr.W, dt))
        q.b.zero_()
        y, got = _product(g, torch, plan, X, q, x32, xp32, 0.3, pen)
        _, again = _product(g, torch, plan, X, q, x32, xp32, 0.3, pen)
        assert np.array_equal(got, again)
        out[prec] = (got, host(q.V))
    got, Vc = out[g.GLAM_BF16]
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    Vp, yp = O.paper_array(Vc), O.paper_array(y)
    ref = O.c_array(O.G(d.Xs, Vp * O.H(d.Xs, yp)))
    scale = O.c_array(_abs_chain(d.Xs, Vp, yp))
    err = np.abs(got - ref)
    assert np.all(err <= 8 * U_BF16 * scale + 1e-5 * scale.max()), float((err / scale).max())
    # the product's relative error in norm, the figure a BF16 product is judged by
    rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert rel <= 1e-2, rel
    assert np.abs(got - out[g.GLAM_FP32][0]).max() > 1e-4 * np.abs(ref).max()


@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON])
def test_bf16_path_polished_to_kkt_1e9_matches_oracle(fam):
    """A masked lambda path with a GLAM_BF16 plan on a tcgen05 shape: the BF16 inner products
    only change iteration counts; the FP64 gradient and KKT test of every outer iteration (the
    polish) take each solution to KKT 1e-9, where it agrees with the oracle's."""
    torch, g = gpu_or_skip()
    from test_gpu_fit import _active_sets_agree, _cast32
    n, p = (64, 32, 9), (7, 9, 5)
    pr = _cast32(gen.random_problem(28, n, p, fam, mask_frac=0.15, basis="normal", pen_w="rand"))
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    lams, thetas, stats, lmax = O.fit_path(d, nlambda=5, ratio=1e-2, tol=1e-11)
    dt = torch.float32
    plan = g.Plan(n, p, fam, g.GLAM_BF16)
    res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                          dev(pr.pen_w, torch.float64), lambdas=list(lams),
                          opts=g.glam_opts_default(tol=1e-9, max_outer=200))
    assert res.status == g.GLAM_OK, res.message
    path = host(res.path)
    for k in range(len(lams)):
        th = O.paper_array(path[k])
        r = O.kkt_residual(d, th, lams[k], lmax)
        assert r <= 1.001e-9, (k, r)
        F, Fref = O.objective(d, th, lams[k]), O.objective(d, thetas[k], lams[k])
        assert abs(F - Fref) <= 1e-10 * abs(Fref), (k, F, Fref)
        same, ndeg = _active_sets_agree(d, th, thetas[k], lams[k], lmax, r + stats[k].kkt)
        assert same, (k, ndeg)


def test_bounded_wait_that_runs_out_is_reported_and_the_plan_stays_usable():
    """glam_opts.wait_limit_s = 0 makes every wait of the tcgen05 kernel give up unless its data
    has already landed: the kernel drains the copies and MMAs it issued, sets its error flag, and
    glam_fit_path returns GLAM_ETIMEOUT.  The same plan then fits the path normally."""
    torch, g = gpu_or_skip()
    n, p = (64, 32, 9), (7, 9, 5)
    pr = gen.random_problem(29, n, p, gen.GAUSSIAN, basis="normal")
    dt = torch.float32
    plan = g.Plan(n, p, gen.GAUSSIAN, g.GLAM_FP32)
    args = ([dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt), dev(pr.pen_w, torch.float64))
    with pytest.raises(g.GlamError) as e:
        g.glam_fit_path(plan, *args, nlambda=3, opts=g.glam_opts_default(wait_limit_s=0.0, lambda_min_ratio=0.1))
    assert e.value.status == g.GLAM_ETIMEOUT, e.value
    res = g.glam_fit_path(plan, *args, nlambda=3, opts=g.glam_opts_default(lambda_min_ratio=0.1))
    assert res.status == g.GLAM_OK, res.message
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    lmax = O.lambda_max(d)
    for k in range(3):
        assert O.kkt_residual(d, O.paper_array(host(res.path[k])), res.lambdas[k], lmax) <= 3e-6
