"""Batched lambda paths (glam_fit_path_batched): many independent fits of uneven shapes and mixed
families on one GPU, each on its own plan.

* Every fit of the batch returns exactly the path the same plan gives when it is fitted alone
  (the batch changes where the kernels run, not their arithmetic), whatever the number of host
  workers;
* every returned solution meets the KKT conditions of Eq. (five), evaluated by the FP64 oracle on
  the FP32-rounded data the GPU saw.
The problems are the first fits of the 64-fit workload (grid sides U{32..96}, p_j U{8..24},
Gaussian or Poisson), with shortened paths.
"""
import numpy as np
import pytest

import gen
import oracle as O
from gpu_helpers import dev, gpu_or_skip, host

pytestmark = pytest.mark.gpu

NFIT = 6
NLAM = 6


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _problems(torch, g):
    probs = gen.make_workload(4, nfit=NFIT)
    out = []
    for pr in probs:
        prec = g.GLAM_FP32
        plan = g.Plan(pr.n, pr.p, pr.family, prec)
        bp = g.BatchProblem(plan, [dev(x, torch.float32) for x in pr.XT], dev(pr.Y, torch.float32),
                            dev(pr.W, torch.float32), dev(pr.pen_w, torch.float64), nlambda=NLAM)
        out.append((pr, bp))
    return out


@pytest.mark.parametrize("threads", [0, 3])
def test_batched_paths_equal_single_fits_and_meet_kkt(threads):
    torch, g = gpu_or_skip()
    pb = _problems(torch, g)
    opts = g.glam_opts_default(tol=1e-6, lambda_min_ratio=1e-2)
    res = g.glam_fit_path_batched([b for _, b in pb], opts=opts, max_threads=threads)
    assert len(res) == NFIT
    for (pr, b), r in zip(pb, res):
        assert r.status == g.GLAM_OK, r.message
        assert r.nfit == NLAM
        alone = g.glam_fit_path(b.plan, b.X, b.Y, b.W, b.pen_w, nlambda=NLAM, opts=opts)
        assert alone.status == g.GLAM_OK
        assert np.array_equal(host(r.path), host(alone.path))
        assert r.lambdas == alone.lambdas
        d = O.GlamData.from_c(pr.family, [_f32(x) for x in pr.XT], _f32(pr.Y), _f32(pr.W), pr.pen_w)
        lmax = O.lambda_max(d)
        assert abs(r.lambdas[0] - lmax) <= 1e-5 * lmax
        path = host(r.path)
        for k in (0, NLAM // 2, NLAM - 1):
            th = O.paper_array(path[k])
            assert O.kkt_residual(d, th, r.lambdas[k], lmax) <= 3e-6, (pr.name, k)


def test_batched_rejects_a_repeated_plan():
    torch, g = gpu_or_skip()
    b0 = _problems(torch, g)[0][1]
    with pytest.raises(g.GlamError) as e:
        g.glam_fit_path_batched([b0, b0])
    assert e.value.status == g.GLAM_EINVAL
