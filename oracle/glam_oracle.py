"""FP64 CPU oracle of the GD-PG penalized GLAM solver -- TEST INFRASTRUCTURE ONLY.

Only the test suite, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may
import this module.  The product path (the CUDA library and its Python binding) never
calls it, and shares no code with it.

It is plain, slow, obviously-correct float64 numpy, written in the paper's notation
(Lund, Vincent & Hansen, "Penalized estimation in large-scale generalized linear array
models"):
  * arrays are indexed as in the paper, A[i1, i2, ..., id], and flattened by `vec`
    (App. A, Eq. index: column-major, i1 fastest);
  * rho, H and G follow App. A and Eqs. (eighteen)/(nineteen) of Sec. 6.1, for one component or
    c > 1 components (GlamData.comps: eta = sum_r H(<X_rj>, Theta_r), theta the concatenation of
    the vec Theta_r, Prop. 1 with the sum over r);
  * the family quantities follow App. B, Eqs. (four), (weights)/(nine) and (tennew);
  * the inner PG (FISTA) loop follows Sec. 3.2 with h and grad h of Eqs.
    (twentyfour)/(twentyfive); the step size is Prop. 1 (Eq. nineteennew);
  * the outer loop is Algorithm 1 (GD-PG) with the Armijo rule of Sec. 5;
  * lambda_max and the warm-started path follow Sec. 6.4.

Library primitives used as steps: numpy tensordot (the contraction inside rho), np.kron
(the explicit tensor-product design, Eq. fivenew), np.linalg.eigvalsh (spectral radius).

Readings where the paper is silent or ambiguous (each also listed in the design notes):
  R1  1/n scaling: F = -(1/n) l + lambda J throughout (the inner problem, Eq. eleven, and the
      Lipschitz constant, Eq. lip, carry 1/n); n counts every cell, masked ones included.
  R2  The IRLS weight includes the observation weight: w_i = a_i theta'(eta_i)(g^-1)'(eta_i),
      z_i = W^-1 u_i + eta_i, and z_i = eta_i where a_i = 0.  The fixed point of the outer
      loop (the PMLE) does not depend on this choice (Sec. 5, remark after the Corollary).
  R3  Gaussian loss f = (1/2n) sum a_i (y_i - eta_i)^2, i.e. -(1/n) l plus the constant
      sum a_i y_i^2 / (2n); Poisson loss f = (1/n) sum a_i (exp(eta_i) - y_i eta_i), i.e.
      -(1/n) l with the constant sum a_i log(y_i!) dropped.
  R4  lambda path: lambda_k = lambda_max * ratio^(k/(K-1)) (log spacing).
  R5  Armijo constants alpha0 = 1, b = 0.5, v = 0.1 (the rule of Sec. 5 leaves them free).
  R6  Inner stop: ||x(l+1) - x(l)||_inf <= tol_inner * max(1, ||x(l)||_inf); outer stop:
      KKT residual <= tol (definition in `kkt_residual`).  The paper gives no criterion.
  R7  Step size delta = 1/L_hat (the package's nu = 1: no inner backtracking).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

GAUSSIAN = 0   # Gaussian, identity link (canonical)
POISSON = 1    # Poisson, log link (canonical)
BINOMIAL = 2   # binomial proportions y in [0, 1] with a_i trials, logit link (canonical)
GAMMA = 3      # Gamma (dispersion 1), log link (not canonical)


# --------------------------------------------------------------------------------------
# App. A: the vec map and rho
# --------------------------------------------------------------------------------------

def vec(A) -> np.ndarray:
    """vec of App. A (Eq. index): column-major flattening, i1 fastest."""
    return np.asarray(A, dtype=np.float64).reshape(-1, order="F")


def unvec(v, shape) -> np.ndarray:
    """Inverse of `vec` for an array of the given paper shape (n1, ..., nd)."""
    return np.asarray(v, dtype=np.float64).reshape(shape, order="F")


def rho(X, A) -> np.ndarray:
    """The rotated H-transform of App. A.

    X is an r x n1 matrix and A an n1 x n2 x ... x nd array; the result is the
    n2 x ... x nd x r array with rho(X, A)[i1, ..., id] = sum_j X[id, j] A[j, i1, ..., i(d-1)]:
    the first mode is contracted with X and the new mode goes last.
    """
    X = np.asarray(X, dtype=np.float64)
    A = np.asarray(A, dtype=np.float64)
    if X.ndim != 2 or X.shape[1] != A.shape[0]:
        raise ValueError(f"rho: X {X.shape} does not match the first mode of A {A.shape}")
    T = np.tensordot(X, A, axes=([1], [0]))   # T[r, i2, ..., id]
    return np.moveaxis(T, 0, -1)               # rotate: new mode last


def H(Xs: Sequence[np.ndarray], Theta) -> np.ndarray:
    """Eq. (eighteen), c = 1: H(<X_j>, Theta) = rho(X_d, ..., rho(X_2, rho(X_1, Theta))).

    Xs[j] is the n_j x p_j marginal design; Theta is p1 x ... x pd; the result is the
    n1 x ... x nd array whose vec is the linear predictor X theta (Eq. seventeen)."""
    A = np.asarray(Theta, dtype=np.float64)
    for X in Xs:
        A = rho(X, A)
    return A


def G(Xs: Sequence[np.ndarray], U) -> np.ndarray:
    """Eq. (nineteen), c = 1: G(<X_j>, U) = rho(X_d^T, ..., rho(X_1^T, U)); vec(G) = X^T vec(U)."""
    A = np.asarray(U, dtype=np.float64)
    for X in Xs:
        A = rho(np.asarray(X).T, A)
    return A


def kron_design(Xs: Sequence[np.ndarray]) -> np.ndarray:
    """The explicit tensor-product design X = X_d (x) ... (x) X_1 of Eq. (fivenew) (tiny sizes)."""
    Phi = np.asarray(Xs[0], dtype=np.float64)
    for X in Xs[1:]:
        Phi = np.kron(np.asarray(X, dtype=np.float64), Phi)
    return Phi


def design_row(Xs, idx) -> np.ndarray:
    """Row [i1, .., id] of X = X_d (x) ... (x) X_1 (Eq. fivenew) as a p1 x .. x pd array, so that
    eta[idx] = sum(design_row * Theta) (one entry of Eq. seventeen without the full product)."""
    r = np.asarray(Xs[0][idx[0]], dtype=np.float64)
    for j in range(1, len(Xs)):
        r = np.kron(np.asarray(Xs[j][idx[j]], dtype=np.float64), r)
    return unvec(r, tuple(X.shape[1] for X in Xs))


def design_col(Xs, midx) -> np.ndarray:
    """Column [j1, .., jd] of X = X_d (x) ... (x) X_1 as an n1 x .. x nd array, so that
    G(U)[midx] = sum(design_col * U)."""
    c = np.asarray(Xs[0][:, midx[0]], dtype=np.float64)
    for j in range(1, len(Xs)):
        c = np.kron(np.asarray(Xs[j][:, midx[j]], dtype=np.float64), c)
    return unvec(c, tuple(X.shape[0] for X in Xs))


# --------------------------------------------------------------------------------------
# App. B: exponential-family quantities (canonical links only: theta(eta) = eta)
# --------------------------------------------------------------------------------------

def _theta(family, eta):
    """The canonical parameter theta(eta) of App. B: eta itself for a canonical link; for the
    Gamma family with log link theta = -1/mu = -exp(-eta)."""
    if family in (GAUSSIAN, POISSON, BINOMIAL):
        return np.asarray(eta, dtype=np.float64).copy()
    if family == GAMMA:
        return -np.exp(-eta)
    raise ValueError(family)


def _canonical_derivative(family, eta):
    """theta'(eta): 1 for the canonical links; exp(-eta) for the Gamma family with log link."""
    if family in (GAUSSIAN, POISSON, BINOMIAL):
        return np.ones_like(eta)
    if family == GAMMA:
        return np.exp(-eta)
    raise ValueError(family)


def _mean(family, eta):
    """g^{-1}(eta)."""
    if family == GAUSSIAN:
        return eta.copy()
    if family in (POISSON, GAMMA):
        return np.exp(eta)
    if family == BINOMIAL:
        return 1.0 / (1.0 + np.exp(-eta))
    raise ValueError(family)


def _mean_derivative(family, eta):
    """(g^{-1})'(eta)."""
    if family == GAUSSIAN:
        return np.ones_like(eta)
    if family in (POISSON, GAMMA):
        return np.exp(eta)
    if family == BINOMIAL:
        mu = _mean(family, eta)
        return mu * (1.0 - mu)
    raise ValueError(family)


def _link_derivative(family, mu):
    """g'(mu)."""
    if family == GAUSSIAN:
        return np.ones_like(mu)
    if family in (POISSON, GAMMA):
        return 1.0 / mu
    if family == BINOMIAL:
        return 1.0 / (mu * (1.0 - mu))
    raise ValueError(family)


def _b(family, th):
    """Log-normaliser b(theta) of the density in App. B (for the Gamma family with dispersion 1,
    b(theta) = -log(-theta))."""
    if family == GAUSSIAN:
        return 0.5 * th * th
    if family == POISSON:
        return np.exp(th)
    if family == BINOMIAL:
        return np.logaddexp(0.0, th)
    if family == GAMMA:
        return -np.log(-th)
    raise ValueError(family)


def mean_response(family, eta):
    """mu = g^{-1}(eta), the mean of y at the linear predictor eta."""
    return _mean(family, eta)


def score(family, eta, y, a):
    """u_i = a_i theta'(eta_i) (y_i - g^{-1}(eta_i)), Eq. (four)."""
    return a * _canonical_derivative(family, eta) * (y - _mean(family, eta))


def irls_weight(family, eta, a):
    """w_i = a_i theta'(eta_i) (g^{-1})'(eta_i): Eq. (weights)/(nine) times a_i (reading R2)."""
    return a * _canonical_derivative(family, eta) * _mean_derivative(family, eta)


def working_response(family, eta, y, a):
    """z = W^{-1} u + eta (Eq. ten); with w from `irls_weight` this is the a-free form of
    Eq. (tennew), z_i = (y_i - mu_i) g'(mu_i) + eta_i; z_i = eta_i where a_i = 0 (R2)."""
    mu = _mean(family, eta)
    z = (y - mu) * _link_derivative(family, mu) + eta
    return np.where(a > 0, z, eta)


def loglik(family, eta, y, a):
    """l(eta) = sum_i a_i (y_i theta(eta_i) - b(theta(eta_i))), Eq. (two)."""
    th = _theta(family, eta)
    return float(np.sum(a * (y * th - _b(family, th))))


def loss(family, eta, y, a) -> float:
    """f(eta) = -(1/n) l(eta) + c, with c = sum a y^2/(2n) for the Gaussian family (reading R3);
    the constants of the other densities (log y!, the binomial coefficients, the Gamma terms in y
    alone) are dropped."""
    n = np.asarray(eta).size
    f = -loglik(family, eta, y, a) / n
    if family == GAUSSIAN:
        f += float(np.sum(a * y * y)) / (2.0 * n)
    return f


def loss_grad_y(family, eta, y, a) -> np.ndarray:
    """df/dy_i of `loss` at fixed eta: Eq. (two) is linear in y with coefficient a_i theta(eta_i),
    so -(1/n) a_i theta(eta_i), plus (1/n) a_i y_i from the Gaussian constant of R3."""
    n = np.asarray(eta).size
    g = -a * _theta(family, eta) / n
    if family == GAUSSIAN:
        g = g + a * y / n
    return g


# --------------------------------------------------------------------------------------
# Penalty and proximal operator (Sec. 6.3)
# --------------------------------------------------------------------------------------

def penalty(theta, pen_w, l1=1.0, l2=0.0) -> float:
    """J(theta) = sum_m omega_m (l1 |theta_m| + l2 theta_m^2): the weighted l1 penalty (l1 = 1,
    l2 = 0), the elastic net ||theta||_1 + alpha ||theta||_2^2 of Sec. 6.3 (l1 = 1, l2 = alpha) and
    the ridge penalty ||theta||_2^2 (l1 = 0, l2 = 1)."""
    t = np.asarray(theta, dtype=np.float64)
    return float(np.sum(pen_w * (l1 * np.abs(t) + l2 * t * t)))


def penalty_prox(z, gamma, l1=1.0, l2=0.0):
    """prox of gamma (l1 |.| + l2 (.)^2) per coordinate (gamma may be per coordinate): the soft
    threshold at gamma l1, then the ridge shrinkage 1 / (1 + 2 gamma l2) (Sec. 6.3)."""
    return soft_threshold(z, gamma * l1) / (1.0 + 2.0 * gamma * l2)


def soft_threshold(z, gamma):
    """prox of gamma*|.|: (|z| - gamma)_+ sign(z) (Sec. 6.3); gamma may be per coordinate."""
    return np.maximum(np.abs(z) - gamma, 0.0) * np.sign(z)


# --------------------------------------------------------------------------------------
# Step size (Prop. 1) and the exact Lipschitz constant (Eq. lip, tiny sizes only)
# --------------------------------------------------------------------------------------

def spectral_radius_gram(X) -> float:
    """varrho(X^T X) for a marginal design X (n_j x p_j)."""
    X = np.asarray(X, dtype=np.float64)
    return float(np.max(np.abs(np.linalg.eigvalsh(X.T @ X))))


def lipschitz_bound(Xs, w) -> float:
    """L_hat = max(w)/n * prod_j varrho(X_j^T X_j), Prop. 1 (Eq. nineteennew) with c = 1."""
    n = np.asarray(w).size
    return float(np.max(w)) / n * math.prod(spectral_radius_gram(X) for X in Xs)


def lipschitz_exact(Xs, w) -> float:
    """L = ||X^T W X||_2 / n, Eq. (lip), from the explicit design (tiny sizes only)."""
    Phi = kron_design(Xs)
    M = Phi.T @ (vec(w)[:, None] * Phi)
    return float(np.linalg.norm(M, 2)) / Phi.shape[0]


# --------------------------------------------------------------------------------------
# Tensor-product weights (Sec. 6.2, Eq. kronweight): W = w_1 (x) ... (x) w_d
# --------------------------------------------------------------------------------------

def tensor_weight_grams(Xs, ws):
    """The p_j x p_j matrices X_j^T diag(w_j) X_j of Eq. (kronweight)."""
    return [np.asarray(X, dtype=np.float64).T @ (np.asarray(w, dtype=np.float64)[:, None] * X)
            for X, w in zip(Xs, ws)]


def xtwx_tensor(Xs, ws, theta) -> np.ndarray:
    """X^T W X theta for W = w_1 (x) ... (x) w_d, as H(<X_j^T W_j X_j>, theta) (Eq. kronweight):
    the array transform of Eq. (eighteen) with the marginal matrices replaced by the weighted
    Gram matrices, so that only p-sized arrays are touched."""
    return H(tensor_weight_grams(Xs, ws), theta)


def lipschitz_tensor(Xs, ws, n) -> float:
    """The exact L = ||X^T W X||_2 / n for tensor-product W: (1/n) prod_j varrho(X_j^T W_j X_j),
    since the spectrum of a Kronecker product is the set of products of the factors' spectra."""
    return math.prod(float(np.max(np.abs(np.linalg.eigvalsh(M)))) for M in tensor_weight_grams(Xs, ws)) / n


def geometric_mean_weights(V, scaled=False):
    """The tensor approximation of a non-tensor weight array of Sec. 6.2: V_hat = v_1 (x) ... (x) v_d
    with v_j(i) = exp( (1/m_j) sum over the other indices of log V  -  log V_bar ), V_bar the
    geometric mean of all of V, i.e. the paper's product of ratios V / V_bar over the slice taken to
    the power 1/m_j.  V is in paper layout (n1 x ... x nd).  Reading (the paper's V is strictly
    positive): the means run over the cells with V > 0 only, m_j being their number in the slice
    (and n their total), and a slice without such a cell gets the factor 1.  scaled=True returns
    V_bar v_1 in place of v_1 (the iwls option "kron2"; "kron1" is the approximation as printed),
    so that the product reproduces any positive tensor-product V exactly."""
    V = np.asarray(V, dtype=np.float64)
    pos = V > 0
    logV = np.where(pos, np.log(np.where(pos, V, 1.0)), 0.0)
    log_bar = float(logV.sum() / pos.sum()) if pos.any() else 0.0
    out = []
    for j in range(V.ndim):
        other = tuple(k for k in range(V.ndim) if k != j)
        cnt = pos.sum(axis=other)
        s = logV.sum(axis=other)
        vj = np.where(cnt > 0, np.exp(np.where(cnt > 0, s / np.maximum(cnt, 1), 0.0) - log_bar), 1.0)
        out.append(vj)
    if scaled:
        out[0] = out[0] * math.exp(log_bar)
    return out


def tensor_array(ws) -> np.ndarray:
    """w_1 (x) ... (x) w_d as an n1 x ... x nd array (paper layout)."""
    A = np.asarray(ws[0], dtype=np.float64)
    for w in ws[1:]:
        A = np.multiply.outer(A, np.asarray(w, dtype=np.float64))
    return A


# --------------------------------------------------------------------------------------
# Problem container in paper layout
# --------------------------------------------------------------------------------------

def paper_array(c_arr) -> np.ndarray:
    """A C-order (n3, n2, n1) array as the paper's n1 x n2 x n3 array (same memory order)."""
    return np.asarray(c_arr, dtype=np.float64).transpose(2, 1, 0)


def c_array(paper_arr) -> np.ndarray:
    """Inverse of `paper_array`: a C-contiguous (n3, n2, n1) array."""
    return np.ascontiguousarray(np.asarray(paper_arr).transpose(2, 1, 0))


@dataclass
class GlamData:
    """A GLAM fitting problem in paper layout: Xs[j] is n_j x p_j, Y and a are n1 x n2 x n3,
    pen_w is p1 x p2 x p3."""
    family: int
    Xs: List[np.ndarray]
    Y: np.ndarray
    a: np.ndarray
    pen_w: np.ndarray
    l1: float = 1.0   # penalty J = sum omega (l1 |theta| + l2 theta^2), see `penalty`
    l2: float = 0.0

    comps: Optional[List[List[np.ndarray]]] = None  # c > 1: the c marginal design lists (Xs unused)

    @property
    def n(self) -> int:
        return int(self.Y.size)

    @property
    def pshape(self):
        if self.comps is not None:
            return (sum(math.prod(X.shape[1] for X in Xr) for Xr in self.comps),)
        return tuple(X.shape[1] for X in self.Xs)

    def H(self, theta) -> np.ndarray:
        """The linear predictor: H(<X_j>, Theta) (Eq. eighteen); with c > 1 components
        sum_r H(<X_rj>, Theta_r), theta the concatenation (vec Theta_1, ..., vec Theta_c)."""
        if self.comps is None:
            return H(self.Xs, theta)
        eta = np.zeros(self.Y.shape)
        off = 0
        for Xr in self.comps:
            pr = tuple(X.shape[1] for X in Xr)
            k = math.prod(pr)
            eta = eta + H(Xr, unvec(theta[off:off + k], pr))
            off += k
        return eta

    def G(self, U) -> np.ndarray:
        """X^T U: G(<X_j>, U) (Eq. nineteen); with c > 1 components the concatenation of the
        components' vec G(<X_rj>, U)."""
        if self.comps is None:
            return G(self.Xs, U)
        return np.concatenate([vec(G(Xr, U)) for Xr in self.comps])

    def rho_sum(self) -> float:
        """sum over the components of prod_j varrho(X_rj^T X_rj), the factor of Prop. 1 (Eq.
        nineteennew)."""
        comps = self.comps if self.comps is not None else [self.Xs]
        return float(sum(math.prod(spectral_radius_gram(X) for X in Xr) for Xr in comps))

    @classmethod
    def from_c_components(cls, family, XTs, Y, W, pen_w):
        """The model with c components from the library's layout: XTs[r][j] is (p_rj, n_j), Y/W
        (n3, n2, n1), pen_w the flat concatenation of the components' (p_r3, p_r2, p_r1) arrays."""
        comps = [[np.asarray(x, dtype=np.float64).T for x in XT] for XT in XTs]
        return cls(int(family), comps[0], paper_array(Y), paper_array(W),
                   np.concatenate([vec(paper_array(np.asarray(pw, dtype=np.float64))) for pw in pen_w])
                   if isinstance(pen_w, (list, tuple)) else np.asarray(pen_w, dtype=np.float64),
                   comps=comps)

    @classmethod
    def from_c(cls, family, XT, Y, W, pen_w):
        """Build from the C-order layout of the library: XT[j] is (p_j, n_j), Y/W are
        (n3, n2, n1), pen_w is (p3, p2, p1)."""
        return cls(int(family), [np.asarray(x, dtype=np.float64).T for x in XT], paper_array(Y),
                   paper_array(W), paper_array(pen_w))


def objective(data: GlamData, theta, lam) -> float:
    """F(theta) = f(eta(theta)) + lambda J(theta), Eq. (five) with the 1/n scaling of R1."""
    eta = data.H(theta)
    return loss(data.family, eta, data.Y, data.a) + lam * penalty(theta, data.pen_w, data.l1, data.l2)


def gradient(data: GlamData, theta) -> np.ndarray:
    """grad f(theta) = -(1/n) X^T u(eta(theta)) (Eq. three), via G (Eq. nineteen)."""
    eta = data.H(theta)
    u = score(data.family, eta, data.Y, data.a)
    return -data.G(u) / data.n


def penalized_gradient(data: GlamData, theta, lam) -> np.ndarray:
    """grad f(theta) + lambda omega (.) sign(theta): the gradient of F (Eq. five) in every
    coordinate with theta_m != 0; where theta_m = 0 it takes sign(0) = 0, one element of the
    subdifferential of the l1 term."""
    return gradient(data, theta) + lam * data.pen_w * np.sign(theta)


def lambda_max(data: GlamData) -> float:
    """The smallest lambda whose solution is zero (Sec. 6.4): max_m |g_m(0)| / (omega_m l1) with
    g(0) the gradient of f at theta = 0 (the KKT condition of Eq. five at zero).  The ridge
    penalty (l1 = 0) has no such lambda; its path starts from the lasso's value (reading R19)."""
    g0 = gradient(data, np.zeros(data.pshape))
    l1 = data.l1 if data.l1 > 0 else 1.0
    return float(np.max(np.abs(g0) / (data.pen_w * l1)))


def lambda_sequence(lmax, nlambda, ratio) -> np.ndarray:
    """lambda_k = lambda_max * ratio^(k/(K-1)), k = 0..K-1 (reading R4)."""
    if nlambda == 1:
        return np.array([lmax])
    return lmax * ratio ** (np.arange(nlambda) / (nlambda - 1))


def kkt_residual(data: GlamData, theta, lam, lmax, grad=None) -> float:
    """Scaled KKT residual of Eq. (five): r = max_m r_m / lambda_max with
    r_m = |g_m + lambda omega_m (l1 sign(theta_m) + 2 l2 theta_m)| if theta_m != 0 and
    r_m = max(0, |g_m| - lambda omega_m l1) if theta_m = 0, g = grad f(theta) (the distance of -g
    to lambda times the subdifferential of J)."""
    g = gradient(data, theta) if grad is None else grad
    thr = lam * data.pen_w
    r = np.where(theta != 0, np.abs(g + thr * (data.l1 * np.sign(theta) + 2.0 * data.l2 * theta)),
                 np.maximum(0.0, np.abs(g) - thr * data.l1))
    return float(np.max(r)) / lmax


# --------------------------------------------------------------------------------------
# Inner PG loop (Sec. 3.2) on the quadratic model h of Eq. (twentyfour)
# --------------------------------------------------------------------------------------

@dataclass
class InnerResult:
    x: np.ndarray
    iters: int
    history: Optional[list] = None


def inner_pg(data: GlamData, V, Z, theta0, delta, lam, tol=1e-12, max_iter=100000,
             keep_history=False) -> InnerResult:
    """Accelerated proximal gradient on h(x) + lambda J(x), h(x) = (1/2n)||sqrt(W)(Xx - z)||^2.

    x(0) = x(1) = theta0, omega_l = (l-1)/(l+2), y = x(l) + omega_l (x(l) - x(l-1)),
    x(l+1) = prox_{delta lambda}(y - delta grad h(y)) with grad h(y) = (1/n) X^T W (X y - z),
    evaluated as (G(V (.) H(y)) - G(V (.) Z)) / n (Eqs. twentyeight and twentysixnew)."""
    n = data.n
    b = data.G(V * Z)
    x_prev = np.array(theta0, dtype=np.float64)
    x = x_prev.copy()
    hist = [x.copy()] if keep_history else None
    gam = delta * lam * data.pen_w
    it = 0
    for l in range(1, max_iter + 1):
        it = l
        omega = (l - 1.0) / (l + 2.0)
        y = x + omega * (x - x_prev)
        grad_h = (data.G(V * data.H(y)) - b) / n
        x_new = penalty_prox(y - delta * grad_h, gam, data.l1, data.l2)
        step = float(np.max(np.abs(x_new - x))) if x.size else 0.0
        scale = max(1.0, float(np.max(np.abs(x))) if x.size else 0.0)
        x_prev, x = x, x_new
        if keep_history:
            hist.append(x.copy())
        if step <= tol * scale:
            break
    return InnerResult(x, it, hist)


# --------------------------------------------------------------------------------------
# Algorithm 1 (GD-PG) with the Armijo rule of Sec. 5
# --------------------------------------------------------------------------------------

@dataclass
class FitStats:
    outer_iters: int = 0
    inner_iters: int = 0
    armijo_backtracks: int = 0
    objective: float = float("nan")
    kkt: float = float("nan")
    converged: bool = False
    objective_trace: list = field(default_factory=list)


def gdpg(data: GlamData, lam, theta0, lmax, tol=1e-9, tol_inner=1e-12, max_outer=100,
         max_inner=100000, alpha0=1.0, b=0.5, v=0.1, max_ls=60, weights="exact"):
    """Algorithm 1 (GD-PG) for one lambda.  weights='exact' uses the IRLS weights of App. B
    (times a, R2); weights='one' uses w_i = a_i (any positive weights keep the fixed point,
    Sec. 5); weights='kron1' / 'kron2' use the geometric-mean tensor approximation of the IRLS
    weights (Sec. 6.2, `geometric_mean_weights`) with z = W^-1 u + eta for those weights (Eq. ten)
    and the exact Lipschitz constant of tensor-product weights.  Returns (theta, FitStats)."""
    fam = data.family
    n = data.n
    rho_prod = data.rho_sum()
    theta = np.array(theta0, dtype=np.float64)
    st = FitStats()
    eta = data.H(theta)
    J = lambda t: penalty(t, data.pen_w, data.l1, data.l2)
    F = loss(fam, eta, data.Y, data.a) + lam * J(theta)
    st.objective_trace.append(F)
    for k in range(max_outer):
        # Step 2: U, V and Z at theta(k)
        u = score(fam, eta, data.Y, data.a)
        Lhat = None
        if weights == "exact":
            w = irls_weight(fam, eta, data.a)
            z = working_response(fam, eta, data.Y, data.a)
        elif weights in ("kron1", "kron2"):
            vs = geometric_mean_weights(irls_weight(fam, eta, data.a), scaled=weights == "kron2")
            w = tensor_array(vs)
            z = u / w + eta
            Lhat = lipschitz_tensor(data.Xs, vs, n)
        else:
            w = data.a.astype(np.float64)
            z = np.where(w > 0, u / np.where(w > 0, w, 1.0) + eta, eta)
        # Step 3: delta = 1 / L_hat (Prop. 1; the exact constant for tensor-product weights)
        if Lhat is None:
            Lhat = float(np.max(w)) / n * rho_prod
        if Lhat <= 0:
            break
        delta = 1.0 / Lhat
        # Step 4: inner PG loop
        inner = inner_pg(data, w, z, theta, delta, lam, tol=tol_inner, max_iter=max_inner)
        st.inner_iters += inner.iters
        theta_t = inner.x
        # Step 5: Armijo line search along d = theta~ - theta
        d = theta_t - theta
        eta_t = data.H(theta_t)
        Delta = -float(np.sum(u * (eta_t - eta))) / n + lam * (J(theta_t) - J(theta))
        alpha = alpha0
        accepted = False
        for j in range(max_ls):
            th = theta + alpha * d
            eta_j = data.H(th)
            F_j = loss(fam, eta_j, data.Y, data.a) + lam * J(th)
            if F_j <= F + alpha * v * Delta:
                accepted = True
                break
            alpha *= b
            st.armijo_backtracks += 1
        st.outer_iters = k + 1
        if not accepted:
            break
        theta, eta, F = th, eta_j, F_j
        st.objective_trace.append(F)
        # Step 6: convergence test
        r = kkt_residual(data, theta, lam, lmax)
        st.kkt = r
        if r <= tol:
            st.converged = True
            break
    st.objective = F
    if not st.converged:
        st.kkt = kkt_residual(data, theta, lam, lmax)
        st.converged = st.kkt <= tol
    return theta, st


# --------------------------------------------------------------------------------------
# SCAD penalty by the multistep adaptive lasso (the package's penalty = "scad", Sec. 6.4)
# --------------------------------------------------------------------------------------

SCAD_A = 3.7


def scad_derivative(t, lam, a=SCAD_A):
    """p'_lambda(|t|) of the SCAD penalty: lambda for |t| <= lambda, (a lambda - |t|)_+ / (a - 1)
    beyond."""
    t = np.abs(np.asarray(t, dtype=np.float64))
    return np.where(t <= lam, lam, np.maximum(a * lam - t, 0.0) / (a - 1.0))


def msa_scad(data: GlamData, lam, theta0, lmax, steps, a=SCAD_A, **kw):
    """One lambda of the SCAD fit by the multistep adaptive lasso: step 0 solves the weighted
    lasso with the base weights omega (data.pen_w); step s solves it with the weights
    omega * p'_lambda(|theta^(s-1)|) / lambda, the local linear approximation of the SCAD penalty
    at the previous step's solution (a weighted l1 problem, so Algorithm 1 solves each step).
    Returns (theta, FitStats of the last step, the last step's weights)."""
    theta = np.array(theta0, dtype=np.float64)
    w = data.pen_w
    st = None
    for s in range(steps):
        if s > 0:
            w = data.pen_w * scad_derivative(theta, lam, a) / lam
        ds = GlamData(data.family, data.Xs, data.Y, data.a, w, comps=data.comps)
        theta, st = gdpg(ds, lam, theta, lmax, **kw)
    return theta, st, w


def scad_path(data: GlamData, lambdas, steps, a=SCAD_A, theta0=None, **kw):
    """Warm-started SCAD path: each lambda starts from the previous lambda's solution."""
    lmax = lambda_max(data)
    theta = np.zeros(data.pshape) if theta0 is None else np.array(theta0, dtype=np.float64)
    thetas, stats, weights = [], [], []
    for lam in lambdas:
        theta, st, w = msa_scad(data, lam, theta, lmax, steps, a, **kw)
        thetas.append(theta.copy())
        stats.append(st)
        weights.append(w)
    return np.array(thetas), stats, weights, lmax


def fit_path(data: GlamData, nlambda=10, ratio=1e-3, lambdas=None, theta0=None, **kw):
    """Warm-started lambda path (Sec. 6.4): lambda_max down to ratio*lambda_max, each fit
    started from the previous solution.  Returns (lambdas, thetas[K, p1, .., pd], stats)."""
    lmax = lambda_max(data)
    lams = lambda_sequence(lmax, nlambda, ratio) if lambdas is None else np.asarray(lambdas, float)
    theta = np.zeros(data.pshape) if theta0 is None else np.array(theta0, dtype=np.float64)
    thetas, stats = [], []
    for lam in lams:
        theta, st = gdpg(data, lam, theta, lmax, **kw)
        thetas.append(theta.copy())
        stats.append(st)
    return lams, np.array(thetas), stats, lmax


# --------------------------------------------------------------------------------------
# C-order conveniences (same layout as the library's arguments)
# --------------------------------------------------------------------------------------

def predict_c(XT, theta_c) -> np.ndarray:
    """eta = H(Theta) for C-order inputs: XT[j] (p_j, n_j), theta (p3, p2, p1) -> (n3, n2, n1)."""
    return c_array(H([np.asarray(x).T for x in XT], paper_array(theta_c)))


def G_c(XT, U_c) -> np.ndarray:
    """G(U) for C-order inputs: U (n3, n2, n1) -> (p3, p2, p1)."""
    return c_array(G([np.asarray(x).T for x in XT], paper_array(U_c)))
