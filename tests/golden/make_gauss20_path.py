"""Write gauss20_path.npz: the oracle's lambda path on the 20x20x20 Gaussian workload.

Calls only `gen` (inputs) and `oracle` (FP64 CPU GD-PG).  Stored values:
  lambdas[10], thetas[10, 8, 8, 8] (C-order, p3 x p2 x p1), objective[10], kkt[10], lmax.
Run from the repository root:  python tests/golden/make_gauss20_path.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import gen  # noqa: E402
import oracle as O  # noqa: E402


def main():
    pr = gen.make_workload(0)
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    lams, thetas, stats, lmax = O.fit_path(d, nlambda=pr.nlambda, ratio=pr.lambda_min_ratio, tol=1e-10)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gauss20_path.npz")
    np.savez_compressed(out, lambdas=lams, lmax=lmax,
                        thetas=np.array([O.c_array(t) for t in thetas]),
                        objective=np.array([s.objective for s in stats]),
                        kkt=np.array([s.kkt for s in stats]),
                        inner_iters=np.array([s.inner_iters for s in stats]))
    print("wrote", out, [s.kkt for s in stats])


if __name__ == "__main__":
    main()
