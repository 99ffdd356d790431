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


# ---- the geometric-mean tensor approximation of non-tensor weights (Sec. 6.2) ----

def test_geometric_mean_weights_hand_example():
    """V = (1, 4) along mode 1: log V_bar = log 2, so v1 = (1/2, 2) as printed (kron1) and
    V_bar v1 = (1, 4) with the mean restored (kron2); the single-index modes get 1."""
    V = np.array([1.0, 4.0]).reshape(2, 1, 1)
    v1, v2, v3 = O.geometric_mean_weights(V)
    assert np.allclose(v1, [0.5, 2.0], rtol=1e-15) and np.allclose(v2, [1.0]) and np.allclose(v3, [1.0])
    w1, w2, w3 = O.geometric_mean_weights(V, scaled=True)
    assert np.allclose(w1, [1.0, 4.0], rtol=1e-15) and np.allclose(w2, [1.0]) and np.allclose(w3, [1.0])


def test_geometric_mean_weights_skip_masked_cells_by_hand():
    """V(i1, i2) = [[1, 0], [4, 16]] (the 0 a masked cell): the positive cells 1, 4, 16 have
    geometric mean 4; slice means of log V (in units of log 2): mode 1 (0, 3), mode 2 (1, 4), so
    v1 = (1/4, 2), v2 = (1/2, 4), and kron2's v1 = (1, 8)."""
    V = np.array([[1.0, 0.0], [4.0, 16.0]]).reshape(2, 2, 1)
    v1, v2, v3 = O.geometric_mean_weights(V)
    assert np.allclose(v1, [0.25, 2.0], rtol=1e-15)
    assert np.allclose(v2, [0.5, 4.0], rtol=1e-15)
    assert np.allclose(v3, [1.0], rtol=1e-15)
    w1, _, _ = O.geometric_mean_weights(V, scaled=True)
    assert np.allclose(w1, [1.0, 8.0], rtol=1e-15)


def test_geometric_mean_weights_reproduce_tensor_products():
    """For a positive tensor product V = c w1 (x) w2 (x) w3 the approximation with the mean restored
    is V itself, the printed one V / V_bar, V_bar the geometric mean of V; and scaling V by s leaves
    the printed factors alone and multiplies the restored one by s."""
    rng = np.random.default_rng(5)
    ws = [rng.uniform(0.2, 3.0, k) for k in (6, 5, 4)]
    V = 2.5 * O.tensor_array(ws)
    Vbar = float(np.exp(np.mean(np.log(V))))
    assert np.allclose(O.tensor_array(O.geometric_mean_weights(V, scaled=True)), V, rtol=1e-13)
    assert np.allclose(O.tensor_array(O.geometric_mean_weights(V)), V / Vbar, rtol=1e-13)
    a = O.geometric_mean_weights(V)
    b = O.geometric_mean_weights(7.0 * V)
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=1e-13)
    c = O.geometric_mean_weights(7.0 * V, scaled=True)
    assert np.allclose(c[0], 7.0 * O.geometric_mean_weights(V, scaled=True)[0], rtol=1e-13)


def test_geometric_mean_weights_of_empty_slice_is_one():
    V = np.ones((3, 2, 2))
    V[1] = 0.0  # every cell of slice 1 of mode 1 masked
    v1, v2, v3 = O.geometric_mean_weights(V)
    assert np.allclose(v1, [1.0, 1.0, 1.0]) and np.allclose(v2, 1.0) and np.allclose(v3, 1.0)


def test_kron_approximated_weights_reach_the_exact_solution():
    """Sec. 5 (any strictly positive weights keep the fixed point): GD-PG with the kron1 and kron2
    approximations of the Poisson IRLS weights of a masked problem stops at the solution of the
    exact weights."""
    import gen
    pr = gen.random_problem(7, (9, 7, 6), (4, 4, 4), gen.POISSON, mask_frac=0.15, basis="normal")
    d = O.GlamData.from_c(pr.family, pr.XT, pr.Y, pr.W, pr.pen_w)
    lmax = O.lambda_max(d)
    lam = 0.05 * lmax
    th0 = np.zeros(d.pshape)
    te, se = O.gdpg(d, lam, th0, lmax, tol=1e-10, weights="exact")
    assert se.converged
    for wts in ("kron1", "kron2"):
        # KKT 1e-8: near 1e-10 the Armijo test of a weight-approximated direction meets the
        # rounding of F, which is flat to 1e-16 there
        tk, sk = O.gdpg(d, lam, th0, lmax, tol=1e-8, weights=wts, max_outer=400)
        assert sk.converged, (wts, sk.kkt)
        assert np.max(np.abs(tk - te)) <= 1e-5 * max(1.0, np.max(np.abs(te))), wts
        assert abs(sk.objective - se.objective) <= 1e-10 * abs(se.objective)
