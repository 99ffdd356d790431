"""Seeded synthetic inputs for the penalized GLAM solver (both the oracle and the CUDA path).

This module only *makes data*: marginal cubic B-spline bases, response arrays, observation
weights and penalty weights shaped like the paper's 3-D smoothing workloads (Sec. 4.1-4.3
and the simulation study of Sec. 6.5).  It contains none of the solver's arithmetic (no
rho/H/G transform, no family score/weight, no prox, no line search).  The one place where a
tensor-product spline surface is evaluated (the noise-free truth of the Gaussian workloads)
is a plain `np.einsum` over the data-generating coefficients, used only to synthesise Y.

Layout conventions (shared by every consumer):
  * A paper array of size n1 x n2 x n3 is flattened column-major by the `vec` map
    (App. A, Eq. index).  In memory that is a C-order array of shape (n3, n2, n1).
  * A marginal design X_j (n_j x p_j, stored column-major as in R) is the C-order array
    X_j^T of shape (p_j, n_j).  Generators return that array and call it `XT[j]`.
  * Theta (p1 x p2 x p3 in the paper) is a C-order array of shape (p3, p2, p1).

Seeds: numpy PCG64 with seed 1510_03298 + workload index.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SEED_BASE = 1510_03298

GAUSSIAN = 0  # Gaussian family, identity link
POISSON = 1   # Poisson family, log link
BINOMIAL = 2  # binomial proportions with a_i trials, logit link
GAMMA = 3     # Gamma family (shape 2), log link


def cubic_bspline_basis(n_j: int, p_j: int) -> np.ndarray:
    """Marginal design Phi_j (n_j x p_j) of cubic B-splines on the grid x_k = k/(n_j-1).

    The paper fits l1-penalized cubic B-spline bases (Sec. 4.1-4.2) but gives no knot rule.
    Reading used here: p_j - 3 equal knot intervals on [0, 1], extended by three knots on
    each side, evaluated with the Cox-de Boor recursion.  Rows sum to one on [0, 1]
    (partition of unity) and each row has at most four non-zeros.
    """
    if p_j < 4:
        raise ValueError("a cubic B-spline basis needs p_j >= 4")
    x = np.linspace(0.0, 1.0, n_j) if n_j > 1 else np.array([0.5])
    h = 1.0 / (p_j - 3)
    t = np.arange(-3, p_j + 1, dtype=np.float64) * h  # p_j + 4 knots, t[3] = 0, t[p_j] = 1
    xx = x[:, None]
    # degree 0: indicator of [t_i, t_{i+1})
    B = ((xx >= t[None, :-1]) & (xx < t[None, 1:])).astype(np.float64)
    for k in range(1, 4):
        nb = B.shape[1] - 1
        left = (xx - t[None, :nb]) / (t[None, k:k + nb] - t[None, :nb])
        right = (t[None, k + 1:k + 1 + nb] - xx) / (t[None, k + 1:k + 1 + nb] - t[None, 1:1 + nb])
        B = left * B[:, :nb] + right * B[:, 1:nb + 1]
    assert B.shape == (n_j, p_j)
    return B


@dataclass
class Problem:
    """One synthetic GLAM fitting problem (c = 1 component, d = 3)."""
    name: str
    family: int
    n: tuple            # (n1, n2, n3)
    p: tuple            # (p1, p2, p3)
    XT: List[np.ndarray]  # XT[j] has shape (p_j, n_j), float64
    Y: np.ndarray       # (n3, n2, n1) float64
    W: np.ndarray       # (n3, n2, n1) float64 observation weights a_i >= 0
    pen_w: np.ndarray   # (p3, p2, p1) float64 penalty weights omega_m > 0
    nlambda: int = 10
    lambda_min_ratio: float = 1e-3
    theta_true: Optional[np.ndarray] = None
    eta_true: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def ncells(self) -> int:
        return int(np.prod(self.n))

    @property
    def ncoef(self) -> int:
        return int(np.prod(self.p))


def _spline_surface(XT, coef):
    """Noise-free tensor-product spline surface sum_{j} B_j1(x1) B_j2(x2) B_j3(x3) coef[j3,j2,j1],
    returned as a C-order (n3, n2, n1) array (data synthesis only)."""
    return np.einsum("ai,bj,ck,cba->kji", XT[0], XT[1], XT[2], coef, optimize=True)


def _bumps(rng, nb, x1, x2):
    A = rng.uniform(1.0, 2.0, nb)
    c = rng.uniform(0.2, 0.8, (nb, 2))
    s = rng.uniform(0.05, 0.15, nb)
    g1 = x1[None, :]
    g2 = x2[:, None]
    out = []
    for b in range(nb):
        out.append(A[b] * np.exp(-((g1 - c[b, 0]) ** 2 + (g2 - c[b, 1]) ** 2) / (2 * s[b] ** 2)))
    return out  # list of (n2, n1)


def gaussian_spline_problem(rng, n, p, density=0.1, noise=1.0, nlambda=10, ratio=1e-3, name="gauss"):
    """Gaussian workload in the style of a 20x20x20 fit: a sparse N(0,1) coefficient array,
    Y = spline surface + N(0, noise^2), W = 1."""
    XT = [cubic_bspline_basis(n[j], p[j]).T.copy() for j in range(3)]
    P = int(np.prod(p))
    k = int(round(density * P))
    theta = np.zeros(P)
    idx = rng.choice(P, size=k, replace=False)
    theta[idx] = rng.standard_normal(k)
    theta = theta.reshape(p[2], p[1], p[0])
    eta = _spline_surface(XT, theta)
    Y = eta + noise * rng.standard_normal(eta.shape)
    W = np.ones_like(Y)
    return Problem(name, GAUSSIAN, tuple(n), tuple(p), XT, Y, W, np.ones((p[2], p[1], p[0])),
                   nlambda, ratio, theta_true=theta, eta_true=eta)


def neuron_like_problem(rng, n=(128, 128, 600), p=(20, 20, 60), noise=0.5, nlambda=50, ratio=1e-3,
                        name="gauss-bumps"):
    """Gaussian smoothing workload shaped like the voltage-sensitive-dye recordings (Sec. 4.2.1):
    five Gaussian bumps in space times a damped sinusoid in time, plus N(0, noise^2)."""
    n1, n2, n3 = n
    x1 = np.linspace(0, 1, n1)
    x2 = np.linspace(0, 1, n2)
    t = np.linspace(0, 1, n3)
    space = sum(_bumps(rng, 5, x1, x2))                       # (n2, n1)
    temporal = np.exp(-2.0 * t) * np.sin(2 * np.pi * 3.0 * t + np.pi / 4)  # (n3,)
    f = temporal[:, None, None] * space[None, :, :]
    Y = f + noise * rng.standard_normal(f.shape)
    XT = [cubic_bspline_basis(n[j], p[j]).T.copy() for j in range(3)]
    return Problem(name, GAUSSIAN, tuple(n), tuple(p), XT, Y, np.ones_like(Y),
                   np.ones((p[2], p[1], p[0])), nlambda, ratio, eta_true=f)


def poisson_log_rate(rng, n, nb=5):
    """Smooth log-rate in [-2, 4]: bumps in space, each modulated by its own sinusoid in time."""
    n1, n2, n3 = n
    x1 = np.linspace(0, 1, n1)
    x2 = np.linspace(0, 1, n2)
    t = np.linspace(0, 1, n3)
    bumps = _bumps(rng, nb, x1, x2)
    k = rng.integers(1, 8, nb)
    phi = rng.uniform(0, 2 * np.pi, nb)
    s = np.zeros((n3, n2, n1))
    for b in range(nb):
        s += bumps[b][None, :, :] * (1.0 + 0.5 * np.sin(2 * np.pi * k[b] * t + phi[b]))[:, None, None]
    return -2.0 + 6.0 * (s - s.min()) / (s.max() - s.min())


def taxi_like_problem(rng, n=(96, 96, 365), p=(30, 30, 40), mask_frac=0.1, nlambda=30, ratio=1e-3,
                      name="poisson-counts"):
    """Poisson counts workload shaped like the binned taxi pickups (Sec. 4.2.2 and 4.3):
    Y ~ Poisson(exp(eta*)), eta* a smooth log-rate in [-2, 4], and a random fraction of the
    cells masked by observation weight 0 (an incompletely observed array)."""
    eta = poisson_log_rate(rng, n)
    Y = rng.poisson(np.exp(eta)).astype(np.float64)
    W = np.ones_like(Y)
    N = Y.size
    m = int(round(mask_frac * N))
    if m > 0:
        W.reshape(-1)[rng.choice(N, size=m, replace=False)] = 0.0
    XT = [cubic_bspline_basis(n[j], p[j]).T.copy() for j in range(3)]
    return Problem(name, POISSON, tuple(n), tuple(p), XT, Y, W, np.ones((p[2], p[1], p[0])),
                   nlambda, ratio, eta_true=eta)


def make_workload(index: int, seed: Optional[int] = None, **overrides):
    """The five synthetic workloads (index 0..4):
      0: Gaussian 20x20x20, p = 8^3, sparse truth, W = 1, 10 lambdas
      1: Gaussian 128x128x600, p = (20,20,60), bumps x damped sinusoid, 50 lambdas
      2: Poisson 96x96x365, p = (30,30,40), log-rate in [-2,4], 10% cells masked, 30 lambdas
      3: Poisson 64x64x64, p = 16^3 (gradient / adjoint checks)
      4: 64 independent fits, sides n_j ~ U{32..96}, p_j ~ U{8..24}, mixed families, 20 lambdas
    """
    rng = np.random.default_rng(SEED_BASE + index if seed is None else seed)
    if index == 0:
        kw = dict(n=(20, 20, 20), p=(8, 8, 8), density=0.1, noise=1.0, nlambda=10, ratio=1e-3,
                  name="gauss-20x20x20")
        kw.update(overrides)
        return gaussian_spline_problem(rng, **kw)
    if index == 1:
        kw = dict(n=(128, 128, 600), p=(20, 20, 60), nlambda=50, name="gauss-128x128x600")
        kw.update(overrides)
        return neuron_like_problem(rng, **kw)
    if index == 2:
        kw = dict(n=(96, 96, 365), p=(30, 30, 40), nlambda=30, name="poisson-96x96x365")
        kw.update(overrides)
        return taxi_like_problem(rng, **kw)
    if index == 3:
        kw = dict(n=(64, 64, 64), p=(16, 16, 16), mask_frac=0.0, nlambda=1, name="poisson-64x64x64")
        kw.update(overrides)
        return taxi_like_problem(rng, **kw)
    if index == 4:
        nfit = overrides.pop("nfit", 64)
        probs = []
        for f in range(nfit):
            fam = POISSON if rng.random() < 0.5 else GAUSSIAN
            n = tuple(int(v) for v in rng.integers(32, 97, 3))
            p = tuple(int(v) for v in rng.integers(8, 25, 3))
            sub = np.random.default_rng(rng.integers(0, 2 ** 63 - 1))
            if fam == GAUSSIAN:
                probs.append(gaussian_spline_problem(sub, n, p, nlambda=20, name=f"batch{f}-gauss"))
            else:
                probs.append(taxi_like_problem(sub, n, p, mask_frac=0.0, nlambda=20, name=f"batch{f}-poisson"))
        return probs
    raise ValueError(f"no workload {index}")


def random_problem(seed: int, n, p, family=GAUSSIAN, mask_frac=0.0, basis="spline", pen_w="ones"):
    """Small random problem for parity tests with odd (ragged) sizes.

    basis='spline' uses cubic B-splines (needs p_j >= 4); basis='normal' draws X_j rows
    from N(0, I) as in the simulation study (Sec. 6.5)."""
    rng = np.random.default_rng(seed)
    if basis == "spline":
        XT = [cubic_bspline_basis(n[j], p[j]).T.copy() for j in range(3)]
    else:
        XT = [rng.standard_normal((n[j], p[j])).T.copy() / np.sqrt(max(n[j], 1)) for j in range(3)]
    W = None
    if family == GAUSSIAN:
        theta = rng.standard_normal((p[2], p[1], p[0])) * (rng.random((p[2], p[1], p[0])) < 0.3)
        eta = _spline_surface(XT, theta)
        Y = eta + 0.5 * rng.standard_normal(eta.shape)
    else:
        eta = 1.5 * np.tanh(_spline_surface(XT, rng.standard_normal((p[2], p[1], p[0])) * 0.7))
        if family == POISSON:
            Y = rng.poisson(np.exp(eta)).astype(np.float64)
        elif family == BINOMIAL:
            # proportions of m_i in {1..8} trials with success probability 1 / (1 + exp(-eta))
            m = rng.integers(1, 9, eta.shape)
            Y = rng.binomial(m, 1.0 / (1.0 + np.exp(-eta))) / m
            W = m.astype(np.float64)
        elif family == GAMMA:
            # Gamma draws of shape 2 and mean exp(eta)
            Y = rng.gamma(2.0, np.exp(eta) / 2.0)
        else:
            raise ValueError(family)
    if W is None:
        W = np.ones_like(Y)
    N = Y.size
    m = int(round(mask_frac * N))
    if m > 0:
        W.reshape(-1)[rng.choice(N, size=m, replace=False)] = 0.0
    if pen_w == "ones":
        pw = np.ones((p[2], p[1], p[0]))
    else:
        pw = rng.uniform(0.5, 1.5, (p[2], p[1], p[0]))
    return Problem(f"random-{seed}", family, tuple(n), tuple(p), XT, Y, W, pw, 5, 1e-2, eta_true=eta)
