"""The band description that the banded mode products take from a marginal design (host side of
glam_opts.exploit_bands; tests/band_form_check.cu drives it on the host, no GPU):

* cubic B-spline bases (every row has at most 4 consecutive nonzeros, first columns nondecreasing)
  are accepted, and X is rebuilt exactly from (start(i), the 4 values of row i);
* for every column j, [lo(j), hi(j)) is exactly the set of rows whose 4-wide window covers j, so
  the adjoint sums over a superset of the rows with X(i, j) != 0 and over nothing else;
* bases with fewer than 4 columns, and a zero row between nonzero rows, keep that form;
* dense rows, a row with 5 spread nonzeros, and first columns that decrease are refused.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
K = 4  # values kept per row


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path_factory.mktemp("band") / "band_form_check"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-std=c++17",
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1510_03298_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "band_form_check.cu"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    return str(exe)


def band_form(driver, X):
    """X is n x p (rows i, columns j); the driver takes X^T row-major."""
    n, p = X.shape
    txt = f"{n} {p}\n" + " ".join(repr(float(v)) for v in X.T.reshape(-1)) + "\n"
    out = subprocess.run([driver], input=txt, capture_output=True, text=True, check=True).stdout.split("\n")
    if out[0] != "banded 1":
        assert out[0] == "banded 0"
        return None
    rows = [ln.split() for ln in out[1:1 + n]]
    cols = [ln.split() for ln in out[1 + n:1 + n + p]]
    start = np.array([int(r[1]) for r in rows])
    val = np.array([[float(v) for v in r[2:]] for r in rows])
    lo = np.array([int(c[1]) for c in cols])
    hi = np.array([int(c[2]) for c in cols])
    return start, val, lo, hi


def _check_form(X, form):
    n, p = X.shape
    start, val, lo, hi = form
    assert np.all(np.diff(start) >= 0) and np.all(start >= 0) and np.all(start <= max(p - K, 0))
    R = np.zeros_like(X)
    for i in range(n):
        for t in range(K):
            if start[i] + t < p:
                R[i, start[i] + t] = val[i, t]
            else:
                assert val[i, t] == 0.0
    assert np.array_equal(R, X)  # exact: the values are copied, not recomputed
    for j in range(p):
        covers = [i for i in range(n) if start[i] <= j < start[i] + K]
        assert list(range(lo[j], hi[j])) == covers, j
        assert set(np.nonzero(X[:, j])[0]) <= set(covers), j


@pytest.mark.parametrize("n,p", [(20, 8), (128, 20), (600, 60), (37, 4), (9, 9), (5, 12)])
def test_bspline_bases_are_banded_and_rebuilt_exactly(driver, n, p):
    X = gen.cubic_bspline_basis(n, p)
    form = band_form(driver, X)
    assert form is not None
    _check_form(X, form)


def test_narrow_bases_and_zero_rows(driver):
    rng = np.random.default_rng(5)
    X = np.zeros((7, 3))
    X[:, 0] = rng.uniform(0.1, 1.0, 7)
    X[3:, 2] = 1.0
    form = band_form(driver, X)  # p < 4: every row fits the window
    assert form is not None
    _check_form(X, form)
    B = gen.cubic_bspline_basis(30, 10)
    B[11, :] = 0.0  # a zero row keeps the previous row's start
    form = band_form(driver, B)
    assert form is not None and form[0][11] == form[0][10]
    _check_form(B, form)


def test_non_banded_designs_are_refused(driver):
    rng = np.random.default_rng(6)
    assert band_form(driver, rng.standard_normal((12, 9))) is None  # dense rows
    X = gen.cubic_bspline_basis(25, 12)
    X[7, 0] = 0.5  # row 7 now spans more than 4 columns
    assert band_form(driver, X) is None
    Y = gen.cubic_bspline_basis(25, 12)[::-1].copy()  # first columns decrease down the rows
    assert band_form(driver, Y) is None
