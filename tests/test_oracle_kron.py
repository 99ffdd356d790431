"""Pins of the tensor-product-weight forms of the oracle (Sec. 6.2, Eq. kronweight).

* X^T W X theta through the weighted Gram matrices equals the brute-force product with the
  explicit design and diag(vec W) (tiny sizes);
* the exact Lipschitz constant of tensor-product weights equals the spectral norm of the
  explicit X^T W X / n, and Prop. 1's bound is not below it;
* for constant weights the Gaussian inner problem with the tensor form is the one of the
  exact form, so a Gaussian fit's gradient at any theta is unchanged;
* a planted mistake (the weights of one mode left out) is caught.
"""
import numpy as np

import oracle as O


def _setup(seed, n=(5, 4, 3), p=(3, 2, 3)):
    rng = np.random.default_rng(seed)
    Xs = [rng.standard_normal((n[j], p[j])) for j in range(3)]
    ws = [rng.uniform(0.2, 2.0, n[j]) for j in range(3)]
    W = np.einsum("i,j,k->ijk", ws[0], ws[1], ws[2])
    theta = rng.standard_normal(p)
    return Xs, ws, W, theta


def test_tensor_gram_product_equals_brute_force():
    for seed in range(4):
        Xs, ws, W, theta = _setup(seed)
        Phi = O.kron_design(Xs)
        ref = Phi.T @ (O.vec(W) * (Phi @ O.vec(theta)))
        got = O.vec(O.xtwx_tensor(Xs, ws, theta))
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_exact_lipschitz_of_tensor_weights():
    Xs, ws, W, _ = _setup(7)
    n = W.size
    L = O.lipschitz_tensor(Xs, ws, n)
    assert np.isclose(L, O.lipschitz_exact(Xs, W), rtol=1e-10)
    assert O.lipschitz_bound(Xs, W) >= L * (1 - 1e-12)


def test_constant_weight_tensor_form_matches_exact_hessian_action():
    Xs, _, _, theta = _setup(11)
    c = 1.7
    n = tuple(X.shape[0] for X in Xs)
    ws = [np.full(n[0], c), np.ones(n[1]), np.ones(n[2])]
    Phi = O.kron_design(Xs)
    ref = c * Phi.T @ (Phi @ O.vec(theta))
    assert np.allclose(O.vec(O.xtwx_tensor(Xs, ws, theta)), ref, rtol=1e-12)


def test_planted_missing_mode_weight_is_caught():
    Xs, ws, W, theta = _setup(13)
    wrong = [ws[0], np.ones_like(ws[1]), ws[2]]
    Phi = O.kron_design(Xs)
    ref = Phi.T @ (O.vec(W) * (Phi @ O.vec(theta)))
    assert not np.allclose(O.vec(O.xtwx_tensor(Xs, wrong, theta)), ref, rtol=1e-6)
