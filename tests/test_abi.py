"""The C-ABI library loads and exports every entry point declared in include/*.h, and its
host-side argument checks answer without a GPU (no compute call is made here)."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(glam_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1510_03298_gb300 import build as b
    b.build()
    import paper_1510_03298_gb300 as g
    return g.load_library()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["glam_predict", "glam_gradient", "glam_loss", "glam_prox_step", "glam_fit_path",
                     "glam_plan_create", "glam_plan_destroy", "glam_quad_build", "glam_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported by libglam.so"


def test_opts_default(lib):
    import paper_1510_03298_gb300 as g
    o = g.glam_opts_default()
    assert o.tol == 1e-6 and o.armijo_alpha0 == 1.0 and o.armijo_b == 0.5 and o.armijo_v == 0.1
    assert o.check_every % 2 == 0 and o.max_inner > 0
    assert lib.glam_opts_default(None) == g.GLAM_EINVAL


def test_plan_create_rejects_bad_arguments(lib):
    import paper_1510_03298_gb300 as g
    h = C.c_void_p()
    bad = [
        (g.GlamDims(4, (C.c_int64 * 3)(5, 5, 5), (C.c_int64 * 3)(4, 4, 4)), g.GLAM_GAUSSIAN_IDENTITY, g.GLAM_FP32),
        (g.GlamDims(3, (C.c_int64 * 3)(0, 5, 5), (C.c_int64 * 3)(4, 4, 4)), g.GLAM_GAUSSIAN_IDENTITY, g.GLAM_FP32),
        (g.GlamDims(2, (C.c_int64 * 3)(5, 5, 3), (C.c_int64 * 3)(4, 4, 1)), g.GLAM_GAUSSIAN_IDENTITY, g.GLAM_FP32),
        (g.GlamDims(3, (C.c_int64 * 3)(5, 5, 5), (C.c_int64 * 3)(4, 4, 4)), 7, g.GLAM_FP32),
        (g.GlamDims(3, (C.c_int64 * 3)(5, 5, 5), (C.c_int64 * 3)(4, 4, 4)), g.GLAM_POISSON_LOG, 9),
    ]
    for dims, fam, prec in bad:
        st = lib.glam_plan_create(C.byref(dims), fam, prec, None, C.byref(h))
        assert st == g.GLAM_EINVAL
        assert h.value is None
        assert len(lib.glam_last_error(None)) > 0
    assert lib.glam_plan_create(None, 0, 0, None, C.byref(h)) == g.GLAM_EINVAL


def test_plan_create_rejects_shapes_past_the_cell_limit(lib):
    """n1 n2 n3 and p1 p2 p3 may not exceed 2^40, including shapes whose int64 product would
    wrap around (2^32 x 2^32 = 2^64 -> 0); the refusal comes before any CUDA call."""
    import paper_1510_03298_gb300 as g
    h = C.c_void_p()
    big = [((1 << 32, 1 << 32, 1), (4, 4, 1)), ((1 << 21, 1 << 20, 1), (4, 4, 1)),
           ((5, 5, 5), (1 << 32, 1 << 32, 2)), ((5, 5, 5), (1 << 41, 1, 1)),
           ((1 << 62, 4, 4), (4, 4, 4))]
    for n, p in big:
        dims = g.GlamDims(3, (C.c_int64 * 3)(*n), (C.c_int64 * 3)(*p))
        assert lib.glam_plan_create(C.byref(dims), g.GLAM_GAUSSIAN_IDENTITY, g.GLAM_FP32, None,
                                    C.byref(h)) == g.GLAM_EINVAL, (n, p)
        assert h.value is None
        assert b"too large" in lib.glam_last_error(None)
    n = (C.c_int64 * 3)(5, 5, 5)
    ps = (C.c_int64 * 6)(1 << 30, 1 << 10, 1, 1 << 30, 1 << 10, 1)  # 2^40 + 2^40 coefficients
    assert lib.glam_plan_create_components(3, n, 2, ps, g.GLAM_GAUSSIAN_IDENTITY, g.GLAM_FP32, None,
                                           C.byref(h)) == g.GLAM_EINVAL
    assert b"too many" in lib.glam_last_error(None)


def test_null_plan_is_an_error_not_a_crash(lib):
    import paper_1510_03298_gb300 as g
    X = (C.c_void_p * 3)(None, None, None)
    assert lib.glam_predict(None, X, None, None) == g.GLAM_EINVAL
    assert b"NULL plan" in lib.glam_last_error(None)
    assert lib.glam_loss(None, X, None, None, None, None) == g.GLAM_EINVAL
    assert lib.glam_plan_destroy(None) == g.GLAM_OK


def test_no_cpu_fallback_without_gpu():
    import torch
    import paper_1510_03298_gb300 as g
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        g.Plan((5, 5, 5), (4, 4, 4), g.GLAM_GAUSSIAN_IDENTITY, g.GLAM_FP32)


def test_batched_fit_checks_its_arguments_without_a_gpu(lib):
    import paper_1510_03298_gb300 as g
    assert lib.glam_fit_path_batched(0, None, None, None, 0) == g.GLAM_OK
    assert lib.glam_fit_path_batched(-1, None, None, None, 0) == g.GLAM_EINVAL
    assert lib.glam_fit_path_batched(2, None, None, None, 0) == g.GLAM_EINVAL
    items = (g.GlamBatchItem * 2)()
    plans = (C.c_void_p * 2)(None, None)
    assert lib.glam_fit_path_batched(2, plans, items, None, 0) == g.GLAM_EINVAL
    assert b"NULL plan" in lib.glam_last_error(None)
    plans = (C.c_void_p * 2)(4096, 4096)  # never dereferenced: the repeat is found first
    assert lib.glam_fit_path_batched(2, plans, items, None, 0) == g.GLAM_EINVAL
    assert b"twice" in lib.glam_last_error(None)
