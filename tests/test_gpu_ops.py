"""Parity of the CUDA transforms and entrywise steps against the FP64 oracle, element by element.

Every entry is held to BAR[prec] (1e-5 FP32, 1e-12 FP64) times its absolute-value chain (the
same computation on absolute values; see gpu_helpers), a bound derived from the arithmetic.

Shapes span several 64 x 64 GEMM tiles and 32-wide slab column tiles with ragged tails, the
fused-kernel limit (p2 <= 32) on both sides, a d = 2 problem, and the full 128x128x600 and
96x96x365 workloads (compared on every entry: the oracle runs them in seconds).
"""
import numpy as np
import pytest

import gen
import oracle as O
from gpu_helpers import (BAR, assert_within, cell_scales, chain_G, chain_H, dev, dtype_of, gpu_or_skip,
                         host, plan_prec)

pytestmark = pytest.mark.gpu

SHAPES = [
    ((37, 29, 13), (9, 7, 6)),       # ragged everything
    ((70, 65, 3), (17, 33, 4)),      # p2 = 33: unfused inner path; n1 > 64 tile
    ((129, 33, 7), (5, 4, 11)),      # n1 = 129: five 32-wide column tiles, one lane valid
    ((8, 9, 130), (4, 5, 20)),       # long mode 3 (split-K over 130 rows)
    ((96, 96, 40), (30, 30, 12)),    # workload-like slab
]


def _problem(seed, n, p, fam=gen.GAUSSIAN, mask=0.0):
    return gen.random_problem(seed, n, p, fam, mask_frac=mask, basis="normal")


# extra shapes for H: several 128-row blocks in i2 with a ragged n1 (scalar stores), p1 = p3
# limits of the FP32 slab kernels, and p3 = 65 (the mode-3 GEMM path)
PREDICT_SHAPES = SHAPES + [
    ((131, 257, 5), (32, 31, 64)),
    ((132, 130, 6), (3, 32, 65)),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,p", PREDICT_SHAPES)
def test_predict(prec, n, p):
    torch, g = gpu_or_skip()
    pr = _problem(1, n, p)
    dt = dtype_of(prec)
    plan = g.Plan(n, p, g.GLAM_GAUSSIAN_IDENTITY, plan_prec(g, prec))
    theta = np.random.default_rng(2).standard_normal((p[2], p[1], p[0]))
    eta = g.glam_predict(plan, [dev(x, dt) for x in pr.XT], dev(theta, dt))
    torch.cuda.synchronize()
    Xs = [x.T for x in pr.XT]
    scale = O.c_array(chain_H(Xs, O.paper_array(theta)))
    assert_within(host(eta), O.predict_c(pr.XT, theta), scale, BAR[prec], what="eta")


def test_predict_two_dimensional():
    torch, g = gpu_or_skip()
    rng = np.random.default_rng(3)
    n, p = (45, 31), (7, 9)
    XT = [rng.standard_normal((p[0], n[0])), rng.standard_normal((p[1], n[1]))]
    theta = rng.standard_normal((1, p[1], p[0]))
    plan = g.Plan(n, p, g.GLAM_GAUSSIAN_IDENTITY, g.GLAM_FP64)
    eta = g.glam_predict(plan, [dev(XT[0], torch.float64), dev(XT[1], torch.float64), None],
                         dev(theta, torch.float64))
    ref = O.predict_c(XT + [np.ones((1, 1))], theta)
    scale = O.c_array(chain_H([x.T for x in XT] + [np.ones((1, 1))], O.paper_array(theta)))
    assert_within(host(eta), ref, scale, BAR["fp64"], what="eta (d = 2)")


FAMILIES = [gen.GAUSSIAN, gen.POISSON, gen.BINOMIAL, gen.GAMMA]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", FAMILIES)
@pytest.mark.parametrize("n,p", SHAPES[:4])
def test_gradient_and_loss(prec, fam, n, p):
    torch, g = gpu_or_skip()
    pr = _problem(4, n, p, fam, mask=0.2)
    dt = dtype_of(prec)
    plan = g.Plan(n, p, fam, plan_prec(g, prec))
    theta = 0.3 * np.random.default_rng(5).standard_normal((p[2], p[1], p[0]))
    X = [dev(x, dt) for x in pr.XT]
    grad, loss = g.glam_gradient(plan, X, dev(theta, dt), dev(pr.Y, dt), dev(pr.W, dt), want_loss=True)
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    th = O.paper_array(theta)
    gref = O.c_array(O.gradient(d, th))
    eta = O.H(d.Xs, th)
    su, _, _ = cell_scales(fam, eta, chain_H(d.Xs, th), d.Y, d.a)
    assert_within(host(grad), gref, O.c_array(chain_G(d.Xs, su)) / d.n, BAR[prec], what="grad")
    fref = O.loss(fam, O.H(d.Xs, th), d.Y, d.a)
    assert abs(loss.item() - fref) <= (1e-12 if prec == "fp64" else 1e-6) * abs(fref)
    l2 = g.glam_loss(plan, X, dev(theta, dt), dev(pr.Y, dt), dev(pr.W, dt))
    assert abs(l2.item() - fref) <= (1e-12 if prec == "fp64" else 1e-6) * abs(fref)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", FAMILIES)
@pytest.mark.parametrize("n,p", [SHAPES[0], SHAPES[1], SHAPES[4]])
def test_quad_build_and_prox_step(prec, fam, n, p):
    torch, g = gpu_or_skip()
    pr = _problem(6, n, p, fam, mask=0.1)
    dt = dtype_of(prec)
    plan = g.Plan(n, p, fam, plan_prec(g, prec))
    rng = np.random.default_rng(7)
    theta_k = 0.2 * rng.standard_normal((p[2], p[1], p[0]))
    X = [dev(x, dt) for x in pr.XT]
    q = g.glam_quad_build(plan, X, dev(theta_k, dt), dev(pr.Y, dt), dev(pr.W, dt))
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    eta = O.H(d.Xs, O.paper_array(theta_k))
    w = O.irls_weight(fam, eta, d.a)
    z = O.working_response(fam, eta, d.Y, d.a)
    b = O.G(d.Xs, w * z)
    su, sw, svz = cell_scales(fam, eta, chain_H(d.Xs, O.paper_array(theta_k)), d.Y, d.a)
    assert_within(host(q.V), O.c_array(w), O.c_array(sw), BAR[prec], what="V")
    assert_within(host(q.VZ), O.c_array(w * z), O.c_array(svz), BAR[prec], what="V (.) Z")
    chain_b = chain_G(d.Xs, svz)
    assert_within(host(q.b), O.c_array(b), O.c_array(chain_b), BAR[prec], what="b = G(V (.) Z)")
    Lhat = O.lipschitz_bound(d.Xs, w)
    assert abs(q.Lhat.item() - Lhat) <= (1e-12 if prec == "fp64" else 1e-6) * Lhat
    # one inner PG step (Sec. 3.2) from (x, x_prev) with omega = 0.4 and delta = 1 / L_hat
    x = theta_k + 0.05 * rng.standard_normal(theta_k.shape)
    xp = theta_k + 0.05 * rng.standard_normal(theta_k.shape)
    lam = 0.3 * O.lambda_max(d)
    omega = 0.4
    xn = g.glam_prox_step(plan, X, q, dev(x, dt), dev(xp, dt), omega, 0.0, lam, dev(pr.pen_w, dt))
    xpa, xppa = O.paper_array(x), O.paper_array(xp)
    y = xpa + omega * (xpa - xppa)
    grad_h = (O.G(d.Xs, w * O.H(d.Xs, y)) - b) / d.n
    delta = 1.0 / Lhat
    ref = O.soft_threshold(y - delta * grad_h, delta * lam * d.pen_w)
    got = O.paper_array(host(xn))
    # values agree within the chain of y - delta grad h (the soft threshold is 1-Lipschitz, so a
    # coordinate that flips to or from zero near the threshold also stays inside it); the FP32
    # floor of 1e-7 of the largest chain entry covers the sums of the mode-3 stages
    chain_prod = chain_G(d.Xs, (np.abs(O.paper_array(host(q.V))) + sw) * chain_H(d.Xs, y))
    chain_x = np.abs(y) + delta * (chain_prod + chain_b) / d.n
    assert_within(got, ref, chain_x, BAR[prec], floor=0.0 if prec == "fp64" else 1e-7, what="x_next")
    zmag = np.abs(y - delta * grad_h) - delta * lam * d.pen_w
    clear = np.abs(zmag) > (1e-9 if prec == "fp64" else 1e-4) * np.abs(y).max()
    assert np.array_equal((got != 0)[clear], (ref != 0)[clear])


@pytest.mark.parametrize("n,p,fam", [((128, 128, 600), (20, 20, 60), gen.GAUSSIAN),
                                     ((96, 96, 365), (30, 30, 40), gen.POISSON)])
def test_full_size_transforms_fp32(n, p, fam):
    """The 128x128x600 and 96x96x365 workloads at full size: every entry of H and of the
    gradient against the oracle (FP64 numpy runs these in seconds)."""
    torch, g = gpu_or_skip()
    pr = gen.make_workload(1 if fam == gen.GAUSSIAN else 2)
    assert pr.n == n
    dt = torch.float32
    plan = g.Plan(n, p, fam, g.GLAM_FP32)
    theta = 0.1 * np.random.default_rng(8).standard_normal((p[2], p[1], p[0]))
    X = [dev(x, dt) for x in pr.XT]
    eta = host(g.glam_predict(plan, X, dev(theta, dt)))
    ref = O.predict_c(pr.XT, theta)
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    th = O.paper_array(theta)
    eta_abs = chain_H(d.Xs, th)
    assert_within(eta, ref, O.c_array(eta_abs), BAR["fp32"], what="eta")
    grad = host(g.glam_gradient(plan, X, dev(theta, dt), dev(pr.Y, dt), dev(pr.W, dt)))
    gref = O.c_array(O.gradient(d, th))
    su, _, _ = cell_scales(fam, O.H(d.Xs, th), eta_abs, d.Y, d.a)
    assert_within(grad, gref, O.c_array(chain_G(d.Xs, su)) / d.n, BAR["fp32"], what="grad")
    # sampled single entries through one design row / column (independent of the oracle's rho)
    rng = np.random.default_rng(9)
    for _ in range(8):
        idx = tuple(int(rng.integers(0, n[j])) for j in range(3))
        e = float(np.sum(O.design_row(d.Xs, idx) * O.paper_array(theta)))
        assert abs(eta[idx[2], idx[1], idx[0]] - e) <= BAR["fp32"] * eta_abs[idx]
