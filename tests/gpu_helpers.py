"""Shared helpers of the GPU parity tests (device transfer, error measures, derived bounds).

Parity bars.  Every comparison with the oracle is element by element against a bound derived
from the arithmetic: the same computation with every factor replaced by its absolute value (the
"absolute-value chain", e.g. |H|(|theta|) for eta = H(theta)) bounds, to first order, the rounding
error that each step contributes relative to the magnitudes it combines.  An entry may differ
from the oracle's by BAR[prec] times its chain: 1e-5 for the FP32 plans (the relative bar of
FP32 mode products) and 1e-12 for FP64 plans.  Where a result has no cancellation the chain equals
|result| and the bound is a plain element-wise relative error.
"""
import numpy as np
import pytest

import oracle as O

# max-norm bars kept for scalar checks (objective and loss values)
TOL = {"fp64": 1e-11, "fp32": 1e-5}
# element-wise bars relative to the absolute-value chain
BAR = {"fp64": 1e-12, "fp32": 1e-5}


def gpu_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1510_03298_gb300 as g
    from paper_1510_03298_gb300 import build as b
    b.build()
    g.load_library()
    return torch, g


def dtype_of(prec):
    import torch
    return torch.float64 if prec == "fp64" else torch.float32


def plan_prec(g, prec):
    return g.GLAM_FP64 if prec == "fp64" else g.GLAM_FP32


def dev(a, dt):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def rel_err(a, ref):
    """Largest absolute error over the largest reference magnitude (a max-norm measure, used only
    where a test reports a figure; parity assertions use `assert_within`)."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = max(np.abs(ref).max(), 1e-300)
    return float(np.abs(a - ref).max() / scale)


def f32_rounded(a):
    """The values an FP32 plan sees: `a` rounded to binary32, returned in float64."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


# ------------------------------------------------------------------ absolute-value chains
def abs_designs(Xs):
    return [np.abs(np.asarray(X, dtype=np.float64)) for X in Xs]


def chain_H(Xs, theta):
    """|H|(|theta|) in paper layout: the magnitude scale of eta = H(theta)."""
    return O.H(abs_designs(Xs), np.abs(theta))


def chain_G(Xs, S):
    """|G|(S) for a non-negative cell array S (paper layout)."""
    return O.G(abs_designs(Xs), np.abs(S))


def cell_scales(family, eta, eta_abs, y, a):
    """Per-cell error scales of the score u, the IRLS weight w and V (.) Z = u + w eta when eta
    carries an error of the order of eta_abs = |H|(|theta|) times the unit roundoff (first order in
    that error, App. B formulas):
      Gaussian  u = a (y - eta):          |a| (|y| + eta_abs);                w = a exactly
      Poisson   u = a (y - mu), w = a mu:  |a| (|y| + mu (1 + eta_abs));      |a| mu (1 + eta_abs)
      binomial  u = a (y - mu), w = a d:   |a| (|y| + mu + d eta_abs);        |a| d (1 + eta_abs)
      Gamma     u = a (y/mu - 1), w = a:   |a| (|y|/mu (1 + eta_abs) + 1);    w = a exactly
    with mu the mean and d = mu (1 - mu).  Returns (su, sw, svz)."""
    aa = np.abs(a)
    ay = np.abs(y)
    if family == O.GAUSSIAN:
        su, sw = aa * (ay + eta_abs), aa.copy()
        svz = su + aa * (np.abs(eta) + eta_abs)
    elif family == O.POISSON:
        mu = np.exp(eta)
        su, sw = aa * (ay + mu * (1.0 + eta_abs)), aa * mu * (1.0 + eta_abs)
        svz = su + sw * np.abs(eta) + aa * mu * eta_abs
    elif family == O.BINOMIAL:
        mu = O.mean_response(family, eta)
        dd = mu * (1.0 - mu)
        su, sw = aa * (ay + mu + dd * eta_abs), aa * dd * (1.0 + eta_abs)
        svz = su + sw * np.abs(eta) + aa * dd * eta_abs
    else:
        ie = np.exp(-eta)
        su, sw = aa * (ay * ie * (1.0 + eta_abs) + 1.0), aa.copy()
        svz = su + aa * (np.abs(eta) + eta_abs)
    return su, sw, svz


def assert_within(got, ref, scale, bar, floor=0.0, what=""):
    """Element-wise |got - ref| <= bar * scale + floor * max(scale)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.asarray(scale, dtype=np.float64)
    assert got.shape == ref.shape == scale.shape, (what, got.shape, ref.shape, scale.shape)
    err = np.abs(got - ref)
    lim = bar * scale + floor * float(scale.max(initial=0.0))
    ok = err <= lim
    if not np.all(ok):
        i = np.unravel_index(int(np.argmax(np.where(lim > 0, err / np.maximum(lim, 1e-300), np.inf))), err.shape)
        raise AssertionError(f"{what}: {int((~ok).sum())} of {err.size} entries exceed the bound; worst at {i}: "
                             f"got {got[i]!r} ref {ref[i]!r} err {err[i]:.3e} bound {lim[i]:.3e} "
                             f"(scale {scale[i]:.3e}, bar {bar:g})")
    return float((err / np.maximum(lim, 1e-300)).max(initial=0.0))
