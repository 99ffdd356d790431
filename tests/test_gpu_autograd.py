"""The differentiable penalized negative log-likelihood (torch.autograd.Function over the C ABI's
glam_penalized_nll) against the FP64 oracle and finite differences.

Workload: the Poisson 64 x 64 x 64 GLAM with cubic B-spline bases p = (16, 16, 16), an FP32 plan,
lambda = 0.1 lambda_max, pen_w = 1, and 1000 draws Theta ~ N(0, 0.1^2).  Per draw:
  * F, dF/dTheta and dF/dY from the GPU (forward and backward through autograd) against the
    oracle's objective (Eq. five), penalized gradient and df/dy, at the FP32 bar (1e-5 relative);
  * 8 random directions in Theta, 32 random coordinates and 4 random directions in Y against
    central finite differences (h = 1e-3) of the FP64 oracle objective;
and on the first 10 draws every coordinate against its central finite difference.  Coordinates
with |theta_m| < 2h are left out of the finite differences (the kink of |theta_m| lies within
the step).  Inputs are rounded to FP32 before both sides see them, so the comparison measures
the arithmetic only.
"""
import numpy as np
import pytest

import gen
import oracle as O
from gpu_helpers import BAR, assert_within, cell_scales, chain_G, chain_H, dev, gpu_or_skip, host

pytestmark = pytest.mark.gpu

H_FD = 1e-3
TOL32 = 1e-5
NDRAWS = 1000


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


class _Setup:
    def __init__(self, torch, g):
        pr = gen.make_workload(3)
        self.XT = [_f32(x) for x in pr.XT]
        self.Y, self.W, self.pw = _f32(pr.Y), _f32(pr.W), _f32(pr.pen_w)
        self.fam = pr.family
        self.n, self.p = pr.n, pr.p
        self.data = O.GlamData.from_c(self.fam, self.XT, self.Y, self.W, self.pw)
        self.lam = 0.1 * O.lambda_max(self.data)
        self.plan = g.Plan(pr.n, pr.p, g.GLAM_POISSON_LOG, g.GLAM_FP32)
        f32 = torch.float32
        self.Xd = [dev(x, f32) for x in self.XT]
        self.Wd, self.pwd = dev(self.W, f32), dev(self.pw, f32)
        self.torch, self.g = torch, g

    def gpu(self, theta_c, Y_c=None):
        torch = self.torch
        T = dev(theta_c, torch.float32).requires_grad_(True)
        Yd = dev(self.Y if Y_c is None else Y_c, torch.float32).requires_grad_(True)
        F = self.g.penalized_nll(self.plan, self.Xd, T, Yd, self.Wd, self.lam, self.pwd)
        F.backward()
        torch.cuda.synchronize()
        return float(F.item()), host(T.grad), host(Yd.grad)

    # --- oracle side (paper layout inside, C-order at the boundary)
    def F(self, theta_c, Y_c=None):
        d = self.data if Y_c is None else O.GlamData.from_c(self.fam, self.XT, Y_c, self.W, self.pw)
        return O.objective(d, O.paper_array(theta_c), self.lam)

    def grads(self, theta_c):
        """The oracle's dF/dTheta and dF/dY and their absolute-value chains (the bounds of
        gpu_helpers: |G|(su)/n + lambda w for Theta, the magnitude of df/dy for Y)."""
        th = O.paper_array(theta_c)
        gT = O.c_array(O.penalized_gradient(self.data, th, self.lam))
        eta = O.H(self.data.Xs, th)
        gY = O.c_array(O.loss_grad_y(self.fam, eta, self.data.Y, self.data.a))
        cT, cY = _vjp_chains(self.data, th, eta, self.lam)
        return gT, gY, cT, cY

    def coord_fd(self, theta_c, eta_c, m):
        """Central difference of F along coordinate m = (m3, m2, m1), evaluated on the cells the
        design column reaches (the loss of every other cell is unchanged by the step)."""
        m3, m2, m1 = m
        rows = [self.XT[0][m1], self.XT[1][m2], self.XT[2][m3]]
        s1, s2, s3 = (np.nonzero(r)[0] for r in rows)
        col = (rows[2][s3][:, None, None] * rows[1][s2][None, :, None] * rows[0][s1][None, None, :])
        blk = np.ix_(s3, s2, s1)
        e, y, a = eta_c[blk], self.Y[blk], self.W[blk]
        scale = e.size / float(np.prod(self.n))
        df = (O.loss(self.fam, e + H_FD * col, y, a) - O.loss(self.fam, e - H_FD * col, y, a)) * scale
        t = theta_c[m]
        dp = self.lam * self.pw[m] * (abs(t + H_FD) - abs(t - H_FD))
        return (df + dp) / (2 * H_FD)


def _vjp_chains(data, th, eta, lam):
    """Element-wise scales of dF/dTheta and dF/dY (C layout): the chain of the gradient of f,
    |G|(su)/n, plus lambda w for the penalty term; |df/dy| evaluated on the chain of eta."""
    ea = chain_H(data.Xs, th)
    su, _, _ = cell_scales(data.family, eta, ea, data.Y, data.a)
    cT = chain_G(data.Xs, su) / data.n + lam * np.abs(data.pen_w)
    aa = np.abs(data.a)
    if data.family == O.GAUSSIAN:
        cY = aa * (np.abs(data.Y) + ea)
    elif data.family == O.GAMMA:
        cY = aa * np.exp(-eta) * (1.0 + ea)
    else:
        cY = aa * ea
    return O.c_array(cT), O.c_array(cY / data.n)


@pytest.fixture(scope="module")
def setup():
    torch, g = gpu_or_skip()
    return _Setup(torch, g)


def test_autograd_matches_oracle_and_finite_differences(setup):
    s = setup
    rng = np.random.default_rng(gen.SEED_BASE + 31)
    P = int(np.prod(s.p))
    worst = dict(F=0.0, gT=0.0, gY=0.0, dirT=0.0, coord=0.0, dirY=0.0)
    for k in range(NDRAWS):
        theta = _f32(rng.normal(0.0, 0.1, (s.p[2], s.p[1], s.p[0])))
        F, gT, gY = s.gpu(theta)
        F_o = s.F(theta)
        gT_o, gY_o, cT, cY = s.grads(theta)
        worst["F"] = max(worst["F"], abs(F - F_o) / abs(F_o))
        # element-wise, relative to each entry's chain: the ratio must stay <= TOL32
        worst["gT"] = max(worst["gT"], TOL32 * assert_within(gT, gT_o, cT, TOL32, what="dF/dTheta"))
        worst["gY"] = max(worst["gY"], TOL32 * assert_within(gY, gY_o, cY, TOL32, what="dF/dY"))
        smooth = np.abs(theta) >= 2 * H_FD
        # random directions in Theta (zero on the coordinates near a kink)
        eta_c = O.predict_c(s.XT, theta)
        for _ in range(8):
            D = rng.standard_normal(theta.shape) * smooth
            D /= np.abs(D).max()  # steps of at most h per coordinate: no kink is crossed
            eD = O.predict_c(s.XT, D)
            fp = O.loss(s.fam, O.paper_array(eta_c + H_FD * eD), s.data.Y, s.data.a)
            fm = O.loss(s.fam, O.paper_array(eta_c - H_FD * eD), s.data.Y, s.data.a)
            pp = O.penalty(theta + H_FD * D, s.pw) - O.penalty(theta - H_FD * D, s.pw)
            fd = (fp - fm + s.lam * pp) / (2 * H_FD)
            err = abs(fd - float(np.sum(gT * D))) / (np.linalg.norm(gT) * np.linalg.norm(D))
            worst["dirT"] = max(worst["dirT"], err)
        # random coordinates away from the kink
        cand = np.flatnonzero(smooth)
        for flat in rng.choice(cand, size=32, replace=False):
            m = np.unravel_index(flat, theta.shape)
            fd = s.coord_fd(theta, eta_c, m)
            worst["coord"] = max(worst["coord"], abs(fd - gT[m]) / np.abs(gT).max())
        # random directions in Y (F is linear in Y for the Poisson loss)
        eta_p = O.paper_array(eta_c)
        for _ in range(4):
            D = O.paper_array(rng.standard_normal(s.Y.shape))
            fd = (O.loss(s.fam, eta_p, s.data.Y + H_FD * D, s.data.a)
                  - O.loss(s.fam, eta_p, s.data.Y - H_FD * D, s.data.a)) / (2 * H_FD)
            D = O.c_array(D)
            err = abs(fd - float(np.sum(gY * D))) / (np.linalg.norm(gY) * np.linalg.norm(D))
            worst["dirY"] = max(worst["dirY"], err)
    for key, v in worst.items():
        assert v <= TOL32, (key, worst)
    assert P == 4096


def test_autograd_every_coordinate_first_draws(setup):
    s = setup
    rng = np.random.default_rng(gen.SEED_BASE + 31)
    for k in range(10):
        theta = _f32(rng.normal(0.0, 0.1, (s.p[2], s.p[1], s.p[0])))
        _, gT, _ = s.gpu(theta)
        eta_c = O.predict_c(s.XT, theta)
        scale = np.abs(gT).max()
        checked = 0
        for flat in np.flatnonzero(np.abs(theta) >= 2 * H_FD):
            m = np.unravel_index(flat, theta.shape)
            assert abs(s.coord_fd(theta, eta_c, m) - gT[m]) <= TOL32 * scale, (k, m)
            checked += 1
        assert checked >= 0.9 * theta.size


@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON, gen.BINOMIAL, gen.GAMMA])
def test_gradcheck_fp64_plan(fam):
    """torch.autograd.gradcheck (its own finite differences in FP64) on a small ragged problem
    with an FP64 plan, masked cells and non-unit penalty weights."""
    torch, g = gpu_or_skip()
    n, p = (9, 7, 5), (4, 5, 4)
    pr = gen.random_problem(81 + fam, n, p, fam, mask_frac=0.2, basis="normal", pen_w="random")
    plan = g.Plan(n, p, fam, g.GLAM_FP64)
    f64 = torch.float64
    X = [dev(x, f64) for x in pr.XT]
    W, pw = dev(pr.W, f64), dev(pr.pen_w, f64)
    rng = np.random.default_rng(5)
    th = rng.standard_normal((p[2], p[1], p[0])) * 0.3
    th[np.abs(th) < 0.05] = 0.1  # keep every coordinate away from the kink of |theta_m|
    T = dev(th, f64).requires_grad_(True)
    Y = dev(pr.Y, f64).requires_grad_(True)

    def fn(T_, Y_):
        return g.penalized_nll(plan, X, T_, Y_, W, 0.05, pw)

    assert torch.autograd.gradcheck(fn, (T, Y), eps=1e-6, atol=1e-9, rtol=1e-6)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON, gen.BINOMIAL, gen.GAMMA])
def test_penalized_nll_ragged_against_oracle(prec, fam):
    """Ragged shapes spanning several GEMM tiles, masked cells, random penalty weights; the raw
    entry point with an explicit upstream gradient g = 2.5 (the VJP scales by it)."""
    torch, g = gpu_or_skip()
    n, p = (70, 37, 13), (9, 7, 6)
    pr = gen.random_problem(91 + fam, n, p, fam, mask_frac=0.2, basis="normal", pen_w="random")
    dt = torch.float64 if prec == "fp64" else torch.float32
    cast = (lambda a: np.asarray(a, np.float64)) if prec == "fp64" else _f32
    XT, Y, W, pw = [cast(x) for x in pr.XT], cast(pr.Y), cast(pr.W), cast(pr.pen_w)
    data = O.GlamData.from_c(fam, XT, Y, W, pw)
    rng = np.random.default_rng(6)
    th = cast(rng.standard_normal((p[2], p[1], p[0])) * 0.3 * (rng.random((p[2], p[1], p[0])) < 0.6))
    lam = 0.2 * O.lambda_max(data)
    plan = g.Plan(n, p, fam, g.GLAM_FP64 if prec == "fp64" else g.GLAM_FP32)
    gout = torch.tensor(2.5, dtype=torch.float64, device="cuda")
    F, gT, gY = g.glam_penalized_nll(plan, [dev(x, dt) for x in XT], dev(th, dt), dev(Y, dt), dev(W, dt),
                                     lam, dev(pw, dt), gout=gout, want_grads=True)
    torch.cuda.synchronize()
    thp = O.paper_array(th)
    tol = 1e-11 if prec == "fp64" else TOL32
    assert abs(F.item() - O.objective(data, thp, lam)) <= tol * abs(O.objective(data, thp, lam))
    eta = O.H(data.Xs, thp)
    cT, cY = _vjp_chains(data, thp, eta, lam)
    assert_within(host(gT), 2.5 * O.c_array(O.penalized_gradient(data, thp, lam)), 2.5 * cT, BAR[prec],
                  what="dF/dTheta")
    assert_within(host(gY), 2.5 * O.c_array(O.loss_grad_y(fam, eta, data.Y, data.a)), 2.5 * cY, BAR[prec],
                  what="dF/dY")


def test_penalized_nll_rejects_bad_calls():
    torch, g = gpu_or_skip()
    n, p = (8, 8, 8), (4, 4, 4)
    plan = g.Plan(n, p, g.GLAM_POISSON_LOG, g.GLAM_FP32)
    f32 = torch.float32
    X = [torch.ones((4, 8), dtype=f32, device="cuda") for _ in range(3)]
    T = torch.zeros((4, 4, 4), dtype=f32, device="cuda")
    Y = torch.ones((8, 8, 8), dtype=f32, device="cuda")
    with pytest.raises(g.GlamError) as e:
        g.glam_penalized_nll(plan, X, T, Y, Y, 0.1, T, want_F=False)
    assert e.value.status == g.GLAM_EINVAL
    with pytest.raises(g.GlamError) as e:
        g.glam_penalized_nll(plan, X, T, Y, Y, -1.0, T)
    assert e.value.status == g.GLAM_EINVAL
