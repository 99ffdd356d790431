"""The allocation-free loss entry point, glam_loss_eta_noalloc, called through the C ABI.

Callers that cannot allocate device memory where they need the objective (a stream being
captured into a CUDA graph, a host that owns all device memory through its own pool, a
real-time path) use this entry point: it keeps its reduction scratch in a fixed array inside
the library instead of plan workspace.  Its result must equal the oracle's loss of the same
linear predictor, and the plan-based glam_loss, on two calls in a row (the scratch is reused
between calls), and the calls must leave the device's free memory unchanged.

This file is collected last on purpose, so that a run stopping at the first failure has run
every other test before it; it also passes on its own in a fresh process.
"""
import ctypes as C
import gc

import numpy as np
import pytest

import gen
import oracle as O
from gpu_helpers import dev, f32_rounded, gpu_or_skip, host

pytestmark = pytest.mark.gpu


def _entry(g):
    lib = g.load_library()
    fn = lib.glam_loss_eta_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                   C.c_void_p]
    return lib, fn


def _terms_abs(fam, eta, y, a):
    """sum_i |a_i| |l_i| bounded term by term (the magnitude that the rounding of the per-cell terms
    scales with): Gaussian a (y - eta)^2 / 2, Poisson a (e^eta + |y eta|), binomial
    a (log(1 + e^eta) + |y eta|), Gamma a (y e^-eta + |eta|)."""
    aa = np.abs(a)
    if fam == gen.GAUSSIAN:
        t = 0.5 * aa * (y - eta) ** 2
    elif fam == gen.POISSON:
        t = aa * (np.exp(eta) + np.abs(y * eta))
    elif fam == gen.BINOMIAL:
        t = aa * (np.logaddexp(0.0, eta) + np.abs(y * eta))
    else:
        t = aa * (np.abs(y) * np.exp(-eta) + np.abs(eta))
    return float(np.sum(t))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("fam", [gen.GAUSSIAN, gen.POISSON, gen.BINOMIAL, gen.GAMMA])
@pytest.mark.parametrize("n,p", [((37, 29, 13), (9, 7, 6)), ((128, 128, 600), (20, 20, 60))])
def test_noalloc_loss_matches_oracle_and_glam_loss_twice(prec, fam, n, p):
    torch, g = gpu_or_skip()
    lib, fn = _entry(g)
    pr = gen.random_problem(41, n, p, fam, mask_frac=0.1, basis="normal")
    dt = torch.float64 if prec == "fp64" else torch.float32
    cast = (lambda a: np.asarray(a, np.float64)) if prec == "fp64" else f32_rounded
    plan = g.Plan(n, p, fam, g.GLAM_FP64 if prec == "fp64" else g.GLAM_FP32)
    X = [dev(x, dt) for x in pr.XT]
    theta = dev(0.2 * np.random.default_rng(42).standard_normal((p[2], p[1], p[0])), dt)
    Y, W = dev(pr.Y, dt), dev(pr.W, dt)
    ref_plan = g.glam_loss(plan, X, theta, Y, W).item()
    eta = g.glam_predict(plan, X, theta)
    # the oracle's loss of exactly the eta, Y and W the entry point reads
    eh, yh, wh = host(eta), cast(pr.Y), cast(pr.W)
    ref = O.loss(fam, O.paper_array(eh), O.paper_array(yh), O.paper_array(wh))
    bound = (1e-14 if prec == "fp64" else 1e-6) * _terms_abs(fam, eh, yh, wh) / eh.size
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for _ in range(2):
        out = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        st = fn(fam, g.GLAM_FP64 if prec == "fp64" else g.GLAM_FP32, eta.numel(), eta.data_ptr(),
                Y.data_ptr(), W.data_ptr(), out.data_ptr(), stream)
        assert st == g.GLAM_OK, lib.glam_last_error(None)
        outs.append(out.item())
    for v in outs:
        assert abs(v - ref) <= bound, (v, ref, bound)
        assert abs(v - ref_plan) <= 2 * bound + (1e-12 if prec == "fp64" else 1e-6) * abs(ref_plan), (v, ref_plan)
    assert outs[0] == outs[1]  # fixed summation order: the same bits on every call
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_poisson_large_eta_is_clamped_like_glam_loss(prec):
    """eta above the exponential's range (e^100 overflows binary32): masked cells (a = 0) add
    exactly zero and unmasked ones the clamped term a (e^c - y eta), c = 80 (FP32) or 700 (FP64),
    as in glam_loss; the result is finite."""
    torch, g = gpu_or_skip()
    lib, fn = _entry(g)
    rng = np.random.default_rng(43)
    n = 4099
    eta = rng.standard_normal(n)
    y = rng.poisson(2.0, n).astype(np.float64)
    a = np.ones(n)
    a[:7] = 0.0
    eta[:7] = 100.0 if prec == "fp32" else 800.0     # masked, beyond the clamp
    eta[7:10] = 90.0 if prec == "fp32" else 750.0    # unmasked, beyond the clamp
    c = 80.0 if prec == "fp32" else 700.0
    dt = torch.float64 if prec == "fp64" else torch.float32
    cast = (lambda v: v) if prec == "fp64" else f32_rounded
    eh, yh, ah = cast(eta), cast(y), cast(a)
    terms = ah * (np.exp(np.minimum(eh, c)) - yh * eh)
    ref = float(np.sum(terms)) / n
    out = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
    ed, yd, ad = dev(eh, dt), dev(yh, dt), dev(ah, dt)  # held until the call has run
    st = fn(gen.POISSON, g.GLAM_FP64 if prec == "fp64" else g.GLAM_FP32, n, ed.data_ptr(), yd.data_ptr(),
            ad.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == g.GLAM_OK
    v = out.item()
    assert np.isfinite(v)
    assert abs(v - ref) <= (1e-14 if prec == "fp64" else 1e-6) * float(np.sum(np.abs(terms))) / n, (v, ref)


def test_noalloc_calls_leave_device_memory_unchanged():
    """After a first call (which looks up the scratch address), further calls allocate nothing:
    the device's free memory and PyTorch's allocator are unchanged around them."""
    torch, g = gpu_or_skip()
    lib, fn = _entry(g)
    n = 1 << 20
    x = torch.linspace(-1.0, 1.0, n, dtype=torch.float32, device="cuda")
    y = torch.ones(n, dtype=torch.float32, device="cuda")
    out = torch.zeros((), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert fn(gen.POISSON, g.GLAM_FP32, n, x.data_ptr(), y.data_ptr(), y.data_ptr(), out.data_ptr(), stream) == g.GLAM_OK
    torch.cuda.synchronize()
    # objects of earlier tests (plans, cached tensor blocks) are released first, and the collector
    # stays off while the calls run, so that nothing else frees device memory in between
    gc.collect()
    torch.cuda.empty_cache()
    torch.cuda.synchronize()
    gc.disable()
    try:
        free0, _ = torch.cuda.mem_get_info()
        alloc0 = torch.cuda.memory_allocated()
        for _ in range(3):
            assert fn(gen.POISSON, g.GLAM_FP32, n, x.data_ptr(), y.data_ptr(), y.data_ptr(), out.data_ptr(),
                      stream) == g.GLAM_OK
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    finally:
        gc.enable()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0, (free0, free1)


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
