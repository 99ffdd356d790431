"""The tensor-product-weight inner loop (iwls = GLAM_IWLS_KRON, Sec. 6.2, Eq. kronweight) against
the oracle and against the exact-weight path.

* the 20 x 20 x 20 Gaussian path (W = 1) reaches the oracle's solutions (the stored oracle path):
  KKT of Eq. (five) evaluated by the oracle, objectives, active sets through the KKT bound;
* a ragged Gaussian problem whose observation weights are a random positive tensor product
  (so M_j = X_j^T diag(w_j) X_j differ from the plain Gram matrices) gives the same solutions as
  the exact-weight path and the oracle's KKT conditions hold;
* the 128 x 128 x 600 workload: every lambda of the kron path meets KKT 1e-6 and its objectives
  equal the exact path's;
* the option is refused where the weights are not a tensor product (Poisson; a masked W);
* the Gamma family (log link: IRLS weight = observation weight) takes the same form.
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
def test_kron_gauss20_path_matches_oracle(prec):
    torch, g = gpu_or_skip()
    pr = gen.make_workload(0)
    gold = np.load(os.path.join(GOLDEN, "gauss20_path.npz"))
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    dt = dtype_of(prec)
    plan = g.Plan(pr.n, pr.p, pr.family, plan_prec(g, prec))
    tol = 1e-9 if prec == "fp64" else 1e-6
    res = g.glam_fit_path(plan, [dev(x, dt) for x in pr.XT], dev(pr.Y, dt), dev(pr.W, dt),
                          dev(pr.pen_w, torch.float64), nlambda=10,
                          opts=g.glam_opts_default(tol=tol, lambda_min_ratio=1e-3, iwls=g.GLAM_IWLS_KRON))
    assert res.status == g.GLAM_OK, res.message
    lmax = float(gold["lmax"])
    path = host(res.path)
    for k in range(10):
        th = O.paper_array(path[k])
        lam = res.lambdas[k]
        r = O.kkt_residual(d, th, lam, lmax)
        assert r <= (1e-9 if prec == "fp64" else 3e-6), (k, r)
        F, Fref = O.objective(d, th, lam), float(gold["objective"][k])
        assert abs(F - Fref) <= (1e-10 if prec == "fp64" else 1e-6) * abs(Fref), (k, F, Fref)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.GAMMA])
def test_kron_tensor_weights_match_exact_path(prec, fam):
    """Gaussian and Gamma/log: both have IRLS weight = observation weight, a tensor product here."""
    torch, g = gpu_or_skip()
    n, p = (37, 29, 13), (9, 7, 6)
    pr = gen.random_problem(21, n, p, fam, basis="normal", pen_w="random")
    rng = np.random.default_rng(22)
    ws = [rng.uniform(0.3, 1.8, n[j]) for j in range(3)]
    W = np.einsum("k,j,i->kji", ws[2], ws[1], ws[0])  # C-order (n3, n2, n1)
    dt = dtype_of(prec)
    cast = (lambda a: np.asarray(a, np.float64)) if prec == "fp64" else (
        lambda a: np.asarray(a, np.float32).astype(np.float64))
    XT, Y, Wc = [cast(x) for x in pr.XT], cast(pr.Y), cast(W)
    d = O.GlamData.from_c(fam, XT, Y, Wc, pr.pen_w)
    tol = (1e-8 if fam == gen.GAMMA else 1e-9) if prec == "fp64" else 1e-6
    paths = []
    for iwls in (g.GLAM_IWLS_EXACT, g.GLAM_IWLS_KRON):
        plan = g.Plan(n, p, fam, plan_prec(g, prec))
        res = g.glam_fit_path(plan, [dev(x, dt) for x in XT], dev(Y, dt), dev(Wc, dt),
                              dev(pr.pen_w, torch.float64), nlambda=6,
                              opts=g.glam_opts_default(tol=tol, lambda_min_ratio=1e-2, iwls=iwls,
                                                       max_outer=200))
        assert res.status == g.GLAM_OK, res.message
        paths.append((res.lambdas, host(res.path)))
    lmax = O.lambda_max(d)
    (lam_e, pe), (lam_k, pk) = paths
    assert np.allclose(lam_e, lam_k, rtol=1e-12)
    for k in range(6):
        te, tk = O.paper_array(pe[k]), O.paper_array(pk[k])
        assert O.kkt_residual(d, tk, lam_k[k], lmax) <= (3 * tol if prec == "fp64" else 3e-6), k
        Fe, Fk = O.objective(d, te, lam_e[k]), O.objective(d, tk, lam_k[k])
        assert abs(Fe - Fk) <= (1e-10 if prec == "fp64" else 1e-7) * abs(Fe), (k, Fe, Fk)


def test_kron_full_size_gaussian_path():
    torch, g = gpu_or_skip()
    pr = gen.make_workload(1)
    f32 = torch.float32
    X = [dev(x, f32) for x in pr.XT]
    Y, W, pen = dev(pr.Y, f32), dev(pr.W, f32), dev(pr.pen_w, torch.float64)
    out = {}
    for iwls in (g.GLAM_IWLS_EXACT, g.GLAM_IWLS_KRON):
        plan = g.Plan(pr.n, pr.p, pr.family, g.GLAM_FP32)
        res = g.glam_fit_path(plan, X, Y, W, pen, nlambda=12,
                              opts=g.glam_opts_default(tol=1e-6, lambda_min_ratio=1e-3, iwls=iwls))
        assert res.status == g.GLAM_OK, res.message
        out[iwls] = res
    e, k = out[g.GLAM_IWLS_EXACT], out[g.GLAM_IWLS_KRON]
    for se, sk in zip(e.stats, k.stats):
        assert sk["kkt"] <= 1e-6
        assert abs(se["objective"] - sk["objective"]) <= 1e-9 * abs(se["objective"])


def test_kron_refused_without_tensor_product_weights():
    torch, g = gpu_or_skip()
    n, p = (11, 9, 7), (4, 4, 4)
    opts = g.glam_opts_default(iwls=g.GLAM_IWLS_KRON)
    for fam, mask in ((gen.POISSON, 0.0), (gen.GAUSSIAN, 0.2)):
        pr = gen.random_problem(31, n, p, fam, mask_frac=mask, basis="normal")
        plan = g.Plan(n, p, fam, g.GLAM_FP32)
        with pytest.raises(g.GlamError) as ex:
            g.glam_fit_path(plan, [dev(x, torch.float32) for x in pr.XT], dev(pr.Y, torch.float32),
                            dev(pr.W, torch.float32), dev(pr.pen_w, torch.float64), nlambda=3, opts=opts)
        assert ex.value.status == g.GLAM_EINVAL
