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

# shapes inside the tensor-core kernel's domain (n1 % 32 == 0, n2 % 8 == 0, p1, p2 <= 32)
TC_SHAPES = [
    ((32, 8, 3), (5, 3, 2)),          # one column group, one row block, one K step
    ((64, 24, 7), (9, 17, 4)),        # 64-column warps, p2 = 17 (three K steps), three row groups
    ((96, 40, 13), (30, 25, 6)),      # 32-column warps (n1 % 64 != 0), four K steps, uneven rows
    ((160, 16, 5), (32, 32, 3)),      # ten 16-row MMA0 tiles, p1 = p2 = 32
    ((128, 128, 160), (20, 20, 12)),  # the 128 x 128 slab, two slabs on some CTAs
]
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

