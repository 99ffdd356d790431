"""The spectral radius that the plan set-up takes for the step size of Prop. 1 (rho(X_j^T X_j),
and rho(X_j^T diag(v_j) X_j) for tensor-product weights) comes from a cyclic Jacobi routine on the
host; here it is compared with LAPACK's symmetric eigensolver (numpy.linalg.eigvalsh) on Gram
matrices of B-spline and normal designs, weighted Grams, random symmetric matrices (indefinite,
so that the largest magnitude may be a negative eigenvalue), repeated eigenvalues, and the
degenerate 1 x 1, diagonal and zero matrices (tests/jacobi_check.cpp, host compiler, no GPU)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path_factory.mktemp("jacobi") / "jacobi_check"
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_1510_03298_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "jacobi_check.cpp"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    return str(exe)


def _radii(driver, mats):
    txt = "".join(f"{A.shape[0]}\n" + " ".join(repr(float(v)) for v in A.reshape(-1)) + "\n" for A in mats)
    out = subprocess.run([driver], input=txt, capture_output=True, text=True, check=True).stdout
    return [float(v) for v in out.split()]


def _cases():
    rng = np.random.default_rng(11)
    mats = []
    for n, p in [(20, 8), (128, 20), (600, 60), (365, 40), (9, 4)]:
        B = gen.cubic_bspline_basis(n, p)
        mats.append(B.T @ B)
        w = rng.uniform(0.2, 3.0, n)
        mats.append(B.T @ (w[:, None] * B))
    for n, p in [(50, 17), (33, 32), (64, 64)]:
        X = rng.standard_normal((n, p)) / np.sqrt(n)
        mats.append(X.T @ X)
    for m in [2, 3, 7, 16, 31, 64]:
        S = rng.standard_normal((m, m))
        mats.append(S + S.T)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    mats.append(Q @ np.diag([5.0] * 4 + [1.0] * 4 + [-2.0] * 4) @ Q.T)  # repeated eigenvalues
    mats.append(Q @ np.diag([-7.0] + [3.0] * 11) @ Q.T)  # the largest magnitude is negative
    mats += [np.array([[2.5]]), np.array([[-3.0]]), np.diag([1.0, 4.0, 2.0]), np.zeros((5, 5))]
    return [0.5 * (A + A.T) for A in mats]


def test_spectral_radius_matches_lapack(driver):
    mats = _cases()
    got = _radii(driver, mats)
    assert len(got) == len(mats)
    for A, r in zip(mats, got):
        ref = float(np.max(np.abs(np.linalg.eigvalsh(A))))
        scale = max(1.0, np.linalg.norm(A, 2)) if A.any() else 1.0
        assert abs(r - ref) <= 1e-12 * scale, (A.shape, r, ref)
