"""Shared helpers of the GPU parity tests (device transfer, error measures, tolerances)."""
import numpy as np
import pytest

# Parity bars: FP64 runs compare to the oracle at ~machine precision of the products; FP32 runs
# at the 1e-5 relative bar of the FP32 mode products.
TOL = {"fp64": 1e-11, "fp32": 1e-5}


def gpu_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1510_03298_gb300 as g
    from paper_1510_03298_gb300 import build as b
    b.build()
    g.load_library()
    return torch, g


def dtype_of(prec):
    import torch
    return torch.float64 if prec == "fp64" else torch.float32


def plan_prec(g, prec):
    return g.GLAM_FP64 if prec == "fp64" else g.GLAM_FP32


def dev(a, dt):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def rel_err(a, ref):
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = max(np.abs(ref).max(), 1e-300)
    return float(np.abs(a - ref).max() / scale)
