"""The allocation-free loss entry point, glam_loss_eta_noalloc, called through the C ABI.

Callers that cannot allocate device memory where they need the objective (a stream being
captured into a CUDA graph, a host that owns all device memory through its own pool, a
real-time path) use this entry point: it keeps its reduction scratch in a fixed array inside
the library instead of plan workspace.  Its result must equal the plan-based glam_loss on the
same problem, on two calls in a row (the scratch is reused between calls).

This file is collected last on purpose, so that a run stopping at the first failure has run
every other test before it; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import gen
from gpu_helpers import dev, gpu_or_skip

pytestmark = pytest.mark.gpu


def _entry(g):
    lib = g.load_library()
    fn = lib.glam_loss_eta_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                   C.c_void_p]
    return lib, fn


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON])
@pytest.mark.parametrize("n,p", [((37, 29, 13), (9, 7, 6)), ((128, 128, 600), (20, 20, 60))])
def test_noalloc_loss_matches_glam_loss_twice(prec, fam, n, p):
    torch, g = gpu_or_skip()
    lib, fn = _entry(g)
    pr = gen.random_problem(41, n, p, fam, mask_frac=0.1, basis="normal")
    dt = torch.float64 if prec == "fp64" else torch.float32
    plan = g.Plan(n, p, fam, g.GLAM_FP64 if prec == "fp64" else g.GLAM_FP32)
    X = [dev(x, dt) for x in pr.XT]
    theta = dev(0.2 * np.random.default_rng(42).standard_normal((p[2], p[1], p[0])), dt)
    Y, W = dev(pr.Y, dt), dev(pr.W, dt)
    ref = g.glam_loss(plan, X, theta, Y, W)
    eta = g.glam_predict(plan, X, theta)
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for _ in range(2):
        out = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        st = fn(fam, g.GLAM_FP64 if prec == "fp64" else g.GLAM_FP32, eta.numel(), eta.data_ptr(),
                Y.data_ptr(), W.data_ptr(), out.data_ptr(), stream)
        assert st == g.GLAM_OK, lib.glam_last_error(None)
        outs.append(out.item())
    tol = 1e-12 if prec == "fp64" else 1e-6
    r = ref.item()
    for v in outs:
        assert abs(v - r) <= tol * abs(r), (v, r)
    assert outs[0] == outs[1]  # fixed summation order: the same bits on every call
    plan.close()


def test_noalloc_rejects_bad_sizes():
    torch, g = gpu_or_skip()
    lib, fn = _entry(g)
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros((), dtype=torch.float64, device="cuda")
    for n in (0, (1 << 40) + 1):
        st = fn(gen.GAUSSIAN, g.GLAM_FP64, n, x.data_ptr(), x.data_ptr(), x.data_ptr(), out.data_ptr(), None)
        assert st == g.GLAM_EINVAL
        assert b"n must be" in lib.glam_last_error(None)
    assert fn(7, g.GLAM_FP64, 4, x.data_ptr(), x.data_ptr(), x.data_ptr(), out.data_ptr(), None) == g.GLAM_EINVAL
