"""Pins of the oracle's array transforms (rho, H, G) against facts other than the oracle.

* Kronecker identity of App. A (Eq. seventeen): vec(H(<X_j>, Theta)) = (X_3 (x) X_2 (x) X_1) vec(Theta),
  with the explicit product built by np.kron -- independent of rho.
* G is the transpose of H (Eq. nineteen): vec(G(U)) = X^T vec(U) and <H Theta, U> = <Theta, G U>.
* The mode order is free (Kronecker algebra): all six contraction orders agree.
* The vec index map of App. A (Eq. index) and the C-order layout used by the library.
"""
import itertools

import numpy as np
import pytest

import oracle as O

SHAPES = [
    ((5, 4, 3), (2, 3, 4)),     # distinct, non-square, p_j > n_j on mode 3
    ((7, 1, 6), (3, 1, 2)),     # n_j = p_j = 1 on the middle mode
    ((1, 9, 4), (4, 2, 5)),     # n_1 = 1 with p_1 = 4
    ((11, 8, 13), (6, 5, 7)),
]


def _rand(rng, n, p):
    Xs = [rng.standard_normal((n[j], p[j])) for j in range(3)]
    return Xs, rng.standard_normal(p)


@pytest.mark.parametrize("n,p", SHAPES)
def test_kron_identity(n, p):
    rng = np.random.default_rng(1)
    Xs, Theta = _rand(rng, n, p)
    Phi = np.kron(Xs[2], np.kron(Xs[1], Xs[0]))
    lhs = O.vec(O.H(Xs, Theta))
    rhs = Phi @ Theta.reshape(-1, order="F")
    assert lhs.shape == (int(np.prod(n)),)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-13, atol=1e-13 * np.abs(rhs).max())


@pytest.mark.parametrize("n,p", SHAPES)
def test_G_is_transpose(n, p):
    rng = np.random.default_rng(2)
    Xs, _ = _rand(rng, n, p)
    U = rng.standard_normal(n)
    Phi = np.kron(Xs[2], np.kron(Xs[1], Xs[0]))
    np.testing.assert_allclose(O.vec(O.G(Xs, U)), Phi.T @ U.reshape(-1, order="F"), rtol=1e-12,
                               atol=1e-12)


@pytest.mark.parametrize("n,p", SHAPES)
def test_adjoint_identity(n, p):
    rng = np.random.default_rng(3)
    Xs, Theta = _rand(rng, n, p)
    U = rng.standard_normal(n)
    lhs = float(np.sum(O.H(Xs, Theta) * U))
    rhs = float(np.sum(Theta * O.G(Xs, U)))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_rho_shape_and_rotation():
    # rho maps an r x n1 matrix and an n1 x n2 x n3 array to an n2 x n3 x r array (App. A)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((7, 3))
    A = rng.standard_normal((3, 4, 5))
    R = O.rho(X, A)
    assert R.shape == (4, 5, 7)
    # one entry written out: rho(X, A)[i1, i2, i3] = sum_j X[i3, j] A[j, i1, i2]
    assert np.isclose(R[2, 3, 6], sum(X[6, j] * A[j, 2, 3] for j in range(3)))


def test_mode_order_invariance():
    """Contracting the three modes in any order gives the same array (the Kronecker factors
    act on separate indices).  Mode products here are written with einsum per axis."""
    rng = np.random.default_rng(5)
    n, p = (6, 5, 4), (3, 4, 2)
    Xs, Theta = _rand(rng, n, p)
    ref = O.H(Xs, Theta)
    specs = {0: "ia,abc->ibc", 1: "jb,abc->ajc", 2: "kc,abc->abk"}
    for order in itertools.permutations(range(3)):
        A = Theta
        for m in order:
            A = np.einsum(specs[m], Xs[m], A)
        np.testing.assert_allclose(A, ref, rtol=1e-12, atol=1e-12)


def test_vec_index_map():
    # [i1, i2, i3] = i1 + n1 (i2 + n2 i3) (0-based form of App. A, Eq. index)
    n = (3, 4, 5)
    A = np.arange(np.prod(n), dtype=float).reshape(n, order="F")
    v = O.vec(A)
    for i1, i2, i3 in [(0, 0, 0), (2, 1, 0), (1, 3, 4), (2, 3, 4)]:
        assert v[i1 + n[0] * (i2 + n[1] * i3)] == A[i1, i2, i3]
    np.testing.assert_array_equal(O.unvec(v, n), A)


def test_c_order_layout_matches_vec():
    """The library's C-order (n3, n2, n1) arrays are vec-ordered in memory."""
    rng = np.random.default_rng(6)
    n, p = (5, 3, 4), (2, 3, 2)
    XT = [rng.standard_normal((p[j], n[j])) for j in range(3)]
    theta_c = rng.standard_normal((p[2], p[1], p[0]))
    Phi = np.kron(XT[2].T, np.kron(XT[1].T, XT[0].T))
    eta_c = O.predict_c(XT, theta_c)
    assert eta_c.shape == (n[2], n[1], n[0]) and eta_c.flags.c_contiguous
    np.testing.assert_allclose(eta_c.ravel(), Phi @ theta_c.ravel(), rtol=1e-13, atol=1e-13)
    U = rng.standard_normal((n[2], n[1], n[0]))
    np.testing.assert_allclose(O.G_c(XT, U).ravel(), Phi.T @ U.ravel(), rtol=1e-12, atol=1e-12)


def test_planted_transpose_is_caught(monkeypatch):
    """A transposed operand inside rho (a plausible slip) breaks the Kronecker pin."""
    rng = np.random.default_rng(7)
    n, p = (4, 4, 4), (4, 4, 4)   # square so that the slip still type-checks
    Xs, Theta = _rand(rng, n, p)
    Phi = np.kron(Xs[2], np.kron(Xs[1], Xs[0]))
    good = O.rho

    def bad(X, A):
        return good(np.asarray(X).T, A)

    monkeypatch.setattr(O.glam_oracle, "rho", bad)
    assert not np.allclose(O.vec(O.glam_oracle.H(Xs, Theta)), Phi @ Theta.reshape(-1, order="F"))


def test_design_row_and_column_entries():
    """One row / column of the explicit Kronecker design gives single entries of H and G."""
    rng = np.random.default_rng(8)
    n, p = (5, 4, 3), (2, 3, 4)
    Xs, Theta = _rand(rng, n, p)
    Phi = np.kron(Xs[2], np.kron(Xs[1], Xs[0]))
    U = rng.standard_normal(n)
    for idx in [(0, 0, 0), (4, 3, 2), (2, 1, 0)]:
        i = idx[0] + n[0] * (idx[1] + n[1] * idx[2])
        assert np.isclose(np.sum(O.design_row(Xs, idx) * Theta), Phi[i] @ Theta.reshape(-1, order="F"))
    for midx in [(0, 0, 0), (1, 2, 3), (1, 0, 2)]:
        m = midx[0] + p[0] * (midx[1] + p[1] * midx[2])
        assert np.isclose(np.sum(O.design_col(Xs, midx) * U), Phi[:, m] @ U.reshape(-1, order="F"))
