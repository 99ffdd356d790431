"""Python binding of libglam, the GD-PG penalized GLAM solver for one GB300 GPU.

Argument marshalling only: every step of the method runs in the CUDA kernels of libglam.so,
reached through its C ABI (include/glam.h) with ctypes.  PyTorch supplies device memory and
streams.  Nothing here computes any part of the method, and there is no CPU fallback: if the
library is not built, or no CUDA device is present, every entry point raises.

Layout (same as the C ABI): a paper array n1 x n2 x n3 is a C-order tensor of shape
(n3, n2, n1); Theta is (p3, p2, p1); the marginal design X_j (n_j x p_j, column-major) is the
C-order tensor of shape (p_j, n_j).  float64 tensors for GLAM_FP64 plans, float32 otherwise.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from dataclasses import dataclass
from typing import List, Optional, Sequence

import torch

__all__ = [
    "GLAM_OK", "GLAM_EINVAL", "GLAM_ENOMEM", "GLAM_ECUDA", "GLAM_ENONFINITE", "GLAM_ENOCONV",
    "GLAM_ETIMEOUT", "GLAM_GAUSSIAN_IDENTITY", "GLAM_POISSON_LOG", "GLAM_BINOMIAL_LOGIT", "GLAM_GAMMA_LOG", "GLAM_FP64", "GLAM_FP32",
    "GLAM_TF32", "GLAM_BF16", "GLAM_IWLS_EXACT", "GLAM_IWLS_KRON", "GLAM_PENALTY_LASSO", "GLAM_PENALTY_SCAD", "GLAM_PENALTY_ENET",
    "GLAM_PENALTY_RIDGE", "GlamError", "Plan", "Quad", "FitResult", "library_path", "load_library",
    "glam_opts_default", "glam_plan_create", "glam_plan_destroy", "glam_predict", "glam_gradient",
    "glam_loss", "glam_quad_build", "glam_prox_step", "glam_fit_path", "glam_launch_count",
    "glam_time_inner_kernels", "glam_penalized_nll", "PenalizedNLL", "penalized_nll",
    "BatchProblem", "glam_fit_path_batched",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_HEADER = os.path.join(os.path.dirname(_HERE), "include", "glam.h")


def _header_constants():
    vals = {}
    with open(_HEADER) as f:
        for line in f:
            m = re.match(r"#define\s+(GLAM_[A-Z0-9_]+)\s+(\d+)", line)
            if m:
                vals[m.group(1)] = int(m.group(2))
    return vals


_K = _header_constants()
GLAM_OK = _K["GLAM_OK"]
GLAM_EINVAL = _K["GLAM_EINVAL"]
GLAM_ENOMEM = _K["GLAM_ENOMEM"]
GLAM_ECUDA = _K["GLAM_ECUDA"]
GLAM_ENONFINITE = _K["GLAM_ENONFINITE"]
GLAM_ENOCONV = _K["GLAM_ENOCONV"]
GLAM_ETIMEOUT = _K["GLAM_ETIMEOUT"]
GLAM_GAUSSIAN_IDENTITY = _K["GLAM_GAUSSIAN_IDENTITY"]
GLAM_POISSON_LOG = _K["GLAM_POISSON_LOG"]
GLAM_BINOMIAL_LOGIT = _K["GLAM_BINOMIAL_LOGIT"]
GLAM_GAMMA_LOG = _K["GLAM_GAMMA_LOG"]
GLAM_FP64 = _K["GLAM_FP64"]
GLAM_FP32 = _K["GLAM_FP32"]
GLAM_TF32 = _K["GLAM_TF32"]
GLAM_BF16 = _K["GLAM_BF16"]
GLAM_IWLS_EXACT = _K["GLAM_IWLS_EXACT"]
GLAM_IWLS_KRON = _K["GLAM_IWLS_KRON"]
GLAM_IWLS_KRON1 = _K["GLAM_IWLS_KRON1"]
GLAM_IWLS_KRON2 = _K["GLAM_IWLS_KRON2"]
GLAM_PENALTY_LASSO = _K["GLAM_PENALTY_LASSO"]
GLAM_PENALTY_SCAD = _K["GLAM_PENALTY_SCAD"]
GLAM_PENALTY_ENET = _K["GLAM_PENALTY_ENET"]
GLAM_PENALTY_RIDGE = _K["GLAM_PENALTY_RIDGE"]


class GlamDims(C.Structure):
    _fields_ = [("d", C.c_int32), ("n", C.c_int64 * 3), ("p", C.c_int64 * 3)]


class GlamQuadC(C.Structure):
    _fields_ = [("V", C.c_void_p), ("VZ", C.c_void_p), ("b", C.c_void_p), ("Lhat", C.c_void_p)]


class GlamOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("lambda_min_ratio", C.c_double), ("inner_forcing", C.c_double),
                ("inner_floor", C.c_double), ("armijo_alpha0", C.c_double), ("armijo_b", C.c_double),
                ("armijo_v", C.c_double), ("max_inner", C.c_int32), ("max_outer", C.c_int32),
                ("max_linesearch", C.c_int32), ("check_every", C.c_int32), ("iwls", C.c_int32),
                ("penalty", C.c_int32), ("steps", C.c_int32), ("exploit_bands", C.c_int32), ("reserved", C.c_int32 * 2),
                ("enet_alpha", C.c_double), ("wait_limit_s", C.c_double), ("nu", C.c_double)]


class GlamBatchItem(C.Structure):
    _fields_ = [("X", C.c_void_p * 3), ("Y", C.c_void_p), ("W", C.c_void_p), ("pen_w", C.c_void_p),
                ("nlambda", C.c_int32), ("lambda_", C.POINTER(C.c_double)), ("Theta0", C.c_void_p),
                ("Theta_path", C.c_void_p), ("stats", C.c_void_p), ("nfit", C.c_int32),
                ("status", C.c_int32)]


class GlamStats(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("objective", C.c_double), ("kkt", C.c_double),
                ("time_ms", C.c_double), ("outer_iters", C.c_int32), ("inner_iters", C.c_int32),
                ("fp64_passes", C.c_int32), ("armijo_backtracks", C.c_int32), ("nnz", C.c_int32),
                ("status", C.c_int32), ("inner_restarts", C.c_int32), ("reserved0", C.c_int32)]


def library_path() -> str:
    return os.path.join(_HERE, "libglam.so")


_LIB = None
_VP = C.c_void_p
_X3 = C.c_void_p * 3
_XP = C.POINTER(C.c_void_p)  # 3 design pointers per component


def load_library():
    """Load libglam.so (raises if it has not been built: there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1510_03298_gb300.build.build()")
    lib = C.CDLL(path)
    sig = {
        "glam_opts_default": (C.c_int, [C.POINTER(GlamOpts)]),
        "glam_plan_create": (C.c_int, [C.POINTER(GlamDims), C.c_int, C.c_int, _VP, C.POINTER(_VP)]),
        "glam_plan_create_components": (C.c_int, [C.c_int, C.POINTER(C.c_int64), C.c_int, C.POINTER(C.c_int64),
                                                  C.c_int, C.c_int, _VP, C.POINTER(_VP)]),
        "glam_plan_destroy": (C.c_int, [_VP]),
        "glam_plan_set_stream": (C.c_int, [_VP, _VP]),
        "glam_last_error": (C.c_char_p, [_VP]),
        "glam_predict": (C.c_int, [_VP, _XP, _VP, _VP]),
        "glam_gradient": (C.c_int, [_VP, _XP, _VP, _VP, _VP, _VP, _VP]),
        "glam_loss": (C.c_int, [_VP, _XP, _VP, _VP, _VP, _VP]),
        "glam_quad_build": (C.c_int, [_VP, _XP, _VP, _VP, _VP, C.POINTER(GlamQuadC)]),
        "glam_prox_step": (C.c_int, [_VP, _XP, C.POINTER(GlamQuadC), _VP, _VP, C.c_double, C.c_double,
                                     C.c_double, _VP, _VP]),
        "glam_fit_path": (C.c_int, [_VP, _XP, _VP, _VP, _VP, C.c_int, C.POINTER(C.c_double),
                                    C.POINTER(GlamOpts), _VP, _VP, C.POINTER(GlamStats),
                                    C.POINTER(C.c_int)]),
        "glam_penalized_nll": (C.c_int, [_VP, _XP, _VP, _VP, _VP, C.c_double, _VP, _VP, _VP, _VP, _VP]),
        "glam_fit_path_batched": (C.c_int, [C.c_int, C.POINTER(_VP), C.POINTER(GlamBatchItem),
                                            C.POINTER(GlamOpts), C.c_int]),
        "glam_launch_count": (C.c_int64, []),
        "glam_kron_weights": (C.c_int, [_VP, _VP, C.c_int, _VP, _VP, _VP]),
        "glam_time_inner_kernels": (C.c_int, [_VP, _XP, C.POINTER(GlamQuadC), C.c_int,
                                              C.POINTER(C.c_double)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class GlamError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"libglam status {status}: {message}")
        self.status = status
        self.message = message


def _check(status: int, plan_handle=None):
    if status != GLAM_OK:
        msg = load_library().glam_last_error(plan_handle)
        raise GlamError(status, msg.decode() if msg else "")


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else t.data_ptr()


def glam_opts_default(**overrides) -> GlamOpts:
    o = GlamOpts()
    _check(load_library().glam_opts_default(C.byref(o)))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Plan:
    """A libglam plan for one problem shape, family and precision (owns the device workspace)."""

    def __init__(self, n: Sequence[int], p: Sequence[int], family: int, precision: int,
                 stream: Optional[torch.cuda.Stream] = None):
        if not torch.cuda.is_available():
            raise RuntimeError("libglam needs a CUDA device; no CPU fallback exists")
        lib = load_library()
        n = tuple(int(v) for v in n)
        p = tuple(int(v) for v in p)
        d = 3
        if len(n) == 2:  # a 2-D GLAM: n3 = p3 = 1 and X[2] may be None
            n, p, d = n + (1,), p + (1,), 2
        self.n, self.p = n, p
        self.family, self.precision = family, precision
        self.dtype = torch.float64 if precision == GLAM_FP64 else torch.float32
        self.device = torch.device("cuda", torch.cuda.current_device())
        dims = GlamDims(d, (C.c_int64 * 3)(*n), (C.c_int64 * 3)(*p))
        h = _VP()
        s = (stream or torch.cuda.current_stream()).cuda_stream
        _check(lib.glam_plan_create(C.byref(dims), family, precision, _VP(s), C.byref(h)), None)
        self._h = h

    @property
    def handle(self):
        return self._h

    @property
    def ncells(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def ncoef(self) -> int:
        return self.p[0] * self.p[1] * self.p[2]

    def _sync_stream(self):
        _check(load_library().glam_plan_set_stream(self._h, _VP(torch.cuda.current_stream().cuda_stream)),
               self._h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().glam_plan_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------- argument checks
    def _arr(self, t, shape, name):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch.Tensor")
        if t.device.type != "cuda":
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device != self.device:
            raise ValueError(f"{name} is on {t.device}, the plan on {self.device}")
        if t.dtype != self.dtype:
            raise TypeError(f"{name} must be {self.dtype}, got {t.dtype}")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return t

    def _X(self, X):
        if len(X) != 3:
            raise ValueError("X must hold three marginal designs (X[2] may be None for d = 2)")
        ptrs = []
        for j in range(3):
            if X[j] is None:
                ptrs.append(None)
                continue
            self._arr(X[j], (self.p[j], self.n[j]), f"X[{j}]")
            ptrs.append(X[j].data_ptr())
        return _X3(*ptrs)

    def cells_shape(self):
        return (self.n[2], self.n[1], self.n[0])

    def coef_shape(self):
        return (self.p[2], self.p[1], self.p[0])


class PlanC(Plan):
    """A plan for the model with c components (Sec. 2, Eq. fivenew): eta = sum_r H(<X_rj>, Theta_r).
    ps lists the c parameter shapes (p_r1, p_r2, p_r3) (two entries each for a 2-D GLAM).  The
    coefficients are the concatenation (vec Theta_1, ..., vec Theta_c), a 1-D tensor of
    sum_r p_r1 p_r2 p_r3 entries, and X is a sequence of c design triples."""

    def __init__(self, n: Sequence[int], ps: Sequence[Sequence[int]], family: int, precision: int,
                 stream: Optional[torch.cuda.Stream] = None):
        if not torch.cuda.is_available():
            raise RuntimeError("libglam needs a CUDA device; no CPU fallback exists")
        lib = load_library()
        n = tuple(int(v) for v in n)
        ps = [tuple(int(v) for v in p) for p in ps]
        d = 3
        if len(n) == 2:
            n, ps, d = n + (1,), [p + (1,) for p in ps], 2
        self.n, self.ps, self.p = n, ps, ps[0]
        self.family, self.precision = family, precision
        self.dtype = torch.float64 if precision == GLAM_FP64 else torch.float32
        self.device = torch.device("cuda", torch.cuda.current_device())
        flat = (C.c_int64 * (3 * len(ps)))(*[v for p in ps for v in p])
        h = _VP()
        s = (stream or torch.cuda.current_stream()).cuda_stream
        _check(lib.glam_plan_create_components(d, (C.c_int64 * 3)(*n), len(ps), flat, family, precision, _VP(s),
                                               C.byref(h)), None)
        self._h = h

    @property
    def ncoef(self) -> int:
        return sum(p[0] * p[1] * p[2] for p in self.ps)

    def coef_shape(self):
        return (self.ncoef,)

    def _X(self, X):
        if len(X) != len(self.ps):
            raise ValueError(f"X must hold {len(self.ps)} design triples")
        ptrs = []
        for r, Xr in enumerate(X):
            if len(Xr) != 3:
                raise ValueError("each component needs three marginal designs (the third may be None for d = 2)")
            for j in range(3):
                if Xr[j] is None:
                    ptrs.append(None)
                    continue
                self._arr(Xr[j], (self.ps[r][j], self.n[j]), f"X[{r}][{j}]")
                ptrs.append(Xr[j].data_ptr())
        return (C.c_void_p * len(ptrs))(*ptrs)


def glam_plan_create(n, p, family, precision=GLAM_FP32, stream=None) -> Plan:
    return Plan(n, p, family, precision, stream)


def glam_plan_destroy(plan: Plan) -> None:
    plan.close()


def glam_predict(plan: Plan, X, Theta, eta=None):
    """eta = H(<X_j>, Theta) (Sec. 6.1, Eq. eighteen)."""
    plan._sync_stream()
    x = plan._X(X)
    plan._arr(Theta, plan.coef_shape(), "Theta")
    if eta is None:
        eta = torch.empty(plan.cells_shape(), dtype=plan.dtype, device=Theta.device)
    plan._arr(eta, plan.cells_shape(), "eta")
    _check(load_library().glam_predict(plan.handle, x, _ptr(Theta), _ptr(eta)), plan.handle)
    return eta


def glam_gradient(plan: Plan, X, Theta, Y, W, grad=None, want_loss=False):
    """grad f(Theta) = -(1/n) X^T u (Eq. three); optionally also f(Theta) as a device double."""
    plan._sync_stream()
    x = plan._X(X)
    plan._arr(Theta, plan.coef_shape(), "Theta")
    plan._arr(Y, plan.cells_shape(), "Y")
    plan._arr(W, plan.cells_shape(), "W")
    if grad is None:
        grad = torch.empty(plan.coef_shape(), dtype=plan.dtype, device=Theta.device)
    plan._arr(grad, plan.coef_shape(), "grad")
    loss = torch.empty((), dtype=torch.float64, device=Theta.device) if want_loss else None
    _check(load_library().glam_gradient(plan.handle, x, _ptr(Theta), _ptr(Y), _ptr(W), _ptr(grad),
                                        _ptr(loss)), plan.handle)
    return (grad, loss) if want_loss else grad


def glam_loss(plan: Plan, X, Theta, Y, W):
    """f(Theta) = -(1/n) l (Eq. two), FP64, as a 0-d CUDA float64 tensor."""
    plan._sync_stream()
    x = plan._X(X)
    plan._arr(Theta, plan.coef_shape(), "Theta")
    plan._arr(Y, plan.cells_shape(), "Y")
    plan._arr(W, plan.cells_shape(), "W")
    out = torch.empty((), dtype=torch.float64, device=Theta.device)
    _check(load_library().glam_loss(plan.handle, x, _ptr(Theta), _ptr(Y), _ptr(W), _ptr(out)),
           plan.handle)
    return out


@dataclass
class Quad:
    """The quadratic model of Sec. 3.2 at an anchor (device tensors)."""
    V: torch.Tensor
    VZ: torch.Tensor
    b: torch.Tensor
    Lhat: torch.Tensor

    def c(self):
        return GlamQuadC(self.V.data_ptr(), self.VZ.data_ptr(), self.b.data_ptr(), self.Lhat.data_ptr())


def glam_quad_build(plan: Plan, X, Theta_k, Y, W, quad: Optional[Quad] = None) -> Quad:
    plan._sync_stream()
    x = plan._X(X)
    plan._arr(Theta_k, plan.coef_shape(), "Theta_k")
    plan._arr(Y, plan.cells_shape(), "Y")
    plan._arr(W, plan.cells_shape(), "W")
    dev = Theta_k.device
    if quad is None:
        quad = Quad(torch.empty(plan.cells_shape(), dtype=plan.dtype, device=dev),
                    torch.empty(plan.cells_shape(), dtype=plan.dtype, device=dev),
                    torch.empty(plan.coef_shape(), dtype=plan.dtype, device=dev),
                    torch.empty((), dtype=torch.float64, device=dev))
    qc = quad.c()
    _check(load_library().glam_quad_build(plan.handle, x, _ptr(Theta_k), _ptr(Y), _ptr(W), C.byref(qc)),
           plan.handle)
    return quad


def glam_prox_step(plan: Plan, X, quad: Quad, x, x_prev, omega: float, delta: float, lam: float,
                   pen_w, x_next=None):
    """One inner PG iteration of Sec. 3.2 (delta <= 0: delta = 1 / quad.Lhat)."""
    plan._sync_stream()
    xs = plan._X(X)
    for t, nm in ((x, "x"), (x_prev, "x_prev"), (pen_w, "pen_w")):
        plan._arr(t, plan.coef_shape(), nm)
    if x_next is None:
        x_next = torch.empty(plan.coef_shape(), dtype=plan.dtype, device=x.device)
    plan._arr(x_next, plan.coef_shape(), "x_next")
    qc = quad.c()
    _check(load_library().glam_prox_step(plan.handle, xs, C.byref(qc), _ptr(x), _ptr(x_prev),
                                         float(omega), float(delta), float(lam), _ptr(pen_w),
                                         _ptr(x_next)), plan.handle)
    return x_next


@dataclass
class FitResult:
    lambdas: List[float]
    path: torch.Tensor          # (nlambda, p3, p2, p1)
    stats: List[dict]
    nfit: int
    status: int
    message: str


def glam_fit_path(plan: Plan, X, Y, W, pen_w, nlambda: int = 10, lambdas=None, opts: Optional[GlamOpts] = None,
                  Theta0=None, path=None) -> FitResult:
    """Warm-started GD-PG lambda path (Alg. 1, Sec. 6.4).  pen_w, Theta0 and the returned path are
    float64 CUDA tensors for every plan precision.  Returns the path even when a lambda fails to
    converge (status GLAM_ENOCONV; rows past nfit are not solutions)."""
    plan._sync_stream()
    x = plan._X(X)
    plan._arr(Y, plan.cells_shape(), "Y")
    plan._arr(W, plan.cells_shape(), "W")
    _p64(pen_w, plan.coef_shape(), "pen_w")
    if Theta0 is not None:
        _p64(Theta0, plan.coef_shape(), "Theta0")
    if lambdas is not None:
        nlambda = len(lambdas)
    lam = (C.c_double * nlambda)(*([-1.0] * nlambda if lambdas is None else [float(v) for v in lambdas]))
    if path is None:
        path = torch.empty((nlambda,) + plan.coef_shape(), dtype=torch.float64, device=Y.device)
    _p64(path, (nlambda,) + plan.coef_shape(), "path")
    st = (GlamStats * nlambda)()
    nfit = C.c_int(0)
    o = opts if opts is not None else glam_opts_default()
    status = load_library().glam_fit_path(plan.handle, x, _ptr(Y), _ptr(W), _ptr(pen_w), nlambda, lam,
                                          C.byref(o), _ptr(Theta0), _ptr(path), st, C.byref(nfit))
    msg = load_library().glam_last_error(plan.handle)
    msg = msg.decode() if msg else ""
    if status not in (GLAM_OK, GLAM_ENOCONV):
        raise GlamError(status, msg)
    return FitResult(list(lam), path, _stats_list(st), nfit.value, status, msg)


def _p64(t, shape, name):
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous with shape {tuple(shape)}")
    return t


def glam_kron_weights(plan: Plan, V, scaled: bool = False):
    """Geometric-mean tensor approximation of a weight array (Sec. 6.2): V is a float64 CUDA
    tensor of the plan's cell shape; returns (v1, v2, v3), float64 CUDA tensors of n1, n2, n3
    entries, with V_hat(i1, i2, i3) = v1(i1) v2(i2) v3(i3) (scaled: times the overall geometric
    mean, the iwls option "kron2"; else as printed, "kron1")."""
    plan._sync_stream()
    _p64(V, plan.cells_shape(), "V")
    n = plan.cells_shape()[::-1]
    vs = [torch.empty(int(n[j]), dtype=torch.float64, device=V.device) for j in range(3)]
    _check(load_library().glam_kron_weights(plan.handle, _ptr(V), 1 if scaled else 0, _ptr(vs[0]), _ptr(vs[1]),
                                            _ptr(vs[2])), plan.handle)
    return tuple(vs)


def glam_launch_count() -> int:
    """Kernels launched through libglam by this process so far (graph nodes included)."""
    return int(load_library().glam_launch_count())


def glam_time_inner_kernels(plan: Plan, X, quad: Quad, reps: int = 50):
    """Mean CUDA-event time (ms) per launch of the four inner-iteration kernels on the plan's
    stream: [fused slab G(V(.)H), mode-3 product, split mode-3 adjoint, prox step]."""
    plan._sync_stream()
    xs = plan._X(X)
    ms = (C.c_double * 4)()
    qc = quad.c()
    _check(load_library().glam_time_inner_kernels(plan.handle, xs, C.byref(qc), int(reps), ms), plan.handle)
    return list(ms)


def glam_penalized_nll(plan: Plan, X, Theta, Y, W, lam: float, pen_w, gout=None, want_F=True,
                       grad_Theta=None, grad_Y=None, want_grads=False):
    """F(Theta) = f(Theta) + lam * sum pen_w |Theta| (Sec. 2, Eq. five, 1/n scaling) and, with
    want_grads, the vector-Jacobian product with the upstream scalar gout (0-d float64 CUDA tensor,
    or None for 1): gout * dF/dTheta and gout * dF/dY.  Returns (F or None, grad_Theta, grad_Y)."""
    plan._sync_stream()
    x = plan._X(X)
    plan._arr(Theta, plan.coef_shape(), "Theta")
    plan._arr(Y, plan.cells_shape(), "Y")
    plan._arr(W, plan.cells_shape(), "W")
    plan._arr(pen_w, plan.coef_shape(), "pen_w")
    dev = Theta.device
    if gout is not None:
        if (not isinstance(gout, torch.Tensor) or gout.dtype != torch.float64 or gout.numel() != 1
                or gout.device.type != "cuda"):
            raise TypeError("gout must be a one-element float64 CUDA tensor")
        gout = gout.contiguous()
    F = torch.empty((), dtype=torch.float64, device=dev) if want_F else None
    if want_grads:
        if grad_Theta is None:
            grad_Theta = torch.empty(plan.coef_shape(), dtype=plan.dtype, device=dev)
        if grad_Y is None:
            grad_Y = torch.empty(plan.cells_shape(), dtype=plan.dtype, device=dev)
    if grad_Theta is not None:
        plan._arr(grad_Theta, plan.coef_shape(), "grad_Theta")
    if grad_Y is not None:
        plan._arr(grad_Y, plan.cells_shape(), "grad_Y")
    _check(load_library().glam_penalized_nll(plan.handle, x, _ptr(Theta), _ptr(Y), _ptr(W), float(lam),
                                             _ptr(pen_w), _ptr(gout), _ptr(F), _ptr(grad_Theta),
                                             _ptr(grad_Y)), plan.handle)
    return F, grad_Theta, grad_Y


class PenalizedNLL(torch.autograd.Function):
    """The penalized negative log-likelihood F(Theta, Y) = f + lam * J as a differentiable torch
    function of Theta and Y.  Both passes run in libglam: the forward pass is H (Eq. eighteen), the
    family loss (App. B) and the penalty; the backward pass is the hand-written adjoint (the
    transposed H-transform G of Eq. nineteen applied to the score, plus the derivative of the
    loss in Y and lam * pen_w * sign(Theta), with sign(0) = 0) scaled by the upstream gradient."""

    @staticmethod
    def forward(ctx, Theta, Y, plan, X, W, lam, pen_w):
        F, _, _ = glam_penalized_nll(plan, X, Theta.detach(), Y.detach(), W, lam, pen_w)
        ctx.plan, ctx.X, ctx.W, ctx.lam, ctx.pen_w = plan, X, W, lam, pen_w
        ctx.save_for_backward(Theta.detach(), Y.detach())
        return F

    @staticmethod
    def backward(ctx, gF):
        Theta, Y = ctx.saved_tensors
        need_t, need_y = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_t or need_y):
            return (None,) * 7
        plan = ctx.plan
        gT = torch.empty(plan.coef_shape(), dtype=plan.dtype, device=Theta.device) if need_t else None
        gY = torch.empty(plan.cells_shape(), dtype=plan.dtype, device=Theta.device) if need_y else None
        glam_penalized_nll(plan, ctx.X, Theta, Y, ctx.W, ctx.lam, ctx.pen_w,
                           gout=gF.to(torch.float64), want_F=False, grad_Theta=gT, grad_Y=gY)
        return gT, gY, None, None, None, None, None


def penalized_nll(plan: Plan, X, Theta, Y, W, lam: float, pen_w):
    """Differentiable F(Theta, Y) (0-d float64 CUDA tensor); see PenalizedNLL."""
    return PenalizedNLL.apply(Theta, Y, plan, X, W, float(lam), pen_w)


@dataclass
class BatchProblem:
    """One fit of a batch: its plan and the arguments of glam_fit_path (device tensors)."""
    plan: Plan
    X: list
    Y: torch.Tensor
    W: torch.Tensor
    pen_w: torch.Tensor
    nlambda: int = 10
    lambdas: Optional[list] = None
    Theta0: Optional[torch.Tensor] = None


def _stats_list(st):
    return [dict(lam=s.lambda_, objective=s.objective, kkt=s.kkt, time_ms=s.time_ms,
                 outer_iters=s.outer_iters, inner_iters=s.inner_iters, fp64_passes=s.fp64_passes,
                 armijo_backtracks=s.armijo_backtracks, nnz=s.nnz, status=s.status,
                 inner_restarts=s.inner_restarts) for s in st]


def glam_fit_path_batched(problems: Sequence[BatchProblem], opts: Optional[GlamOpts] = None,
                          max_threads: int = 0) -> List[FitResult]:
    """Independent lambda paths of many problems run concurrently (glam_fit_path_batched).  Each
    problem needs its own plan.  Returns one FitResult per problem (status GLAM_ENOCONV results
    included); raises GlamError for argument errors and for failures other than ENOCONV."""
    lib = load_library()
    n = len(problems)
    items = (GlamBatchItem * n)()
    plans = (_VP * n)()
    keep = []
    for i, pb in enumerate(problems):
        pl = pb.plan
        pl._sync_stream()
        x = pl._X(pb.X)
        pl._arr(pb.Y, pl.cells_shape(), "Y")
        pl._arr(pb.W, pl.cells_shape(), "W")
        _p64(pb.pen_w, pl.coef_shape(), "pen_w")
        if pb.Theta0 is not None:
            _p64(pb.Theta0, pl.coef_shape(), "Theta0")
        nl = len(pb.lambdas) if pb.lambdas is not None else pb.nlambda
        lam = (C.c_double * nl)(*([-1.0] * nl if pb.lambdas is None else [float(v) for v in pb.lambdas]))
        path = torch.empty((nl,) + pl.coef_shape(), dtype=torch.float64, device=pb.Y.device)
        st = (GlamStats * nl)()
        keep.append((lam, path, st))
        it = items[i]
        for j in range(3):
            it.X[j] = x[j]
        it.Y, it.W, it.pen_w = _ptr(pb.Y), _ptr(pb.W), _ptr(pb.pen_w)
        it.nlambda = nl
        it.lambda_ = C.cast(lam, C.POINTER(C.c_double))
        it.Theta0 = _ptr(pb.Theta0)
        it.Theta_path = path.data_ptr()
        it.stats = C.cast(st, C.c_void_p)
        plans[i] = pl.handle
    o = opts if opts is not None else glam_opts_default()
    status = lib.glam_fit_path_batched(n, plans, items, C.byref(o), int(max_threads))
    if status == GLAM_EINVAL and all(it.status == 0 and it.nfit == 0 for it in items):
        msg = lib.glam_last_error(None)
        raise GlamError(status, msg.decode() if msg else "")
    out = []
    for i, pb in enumerate(problems):
        lam, path, st = keep[i]
        it = items[i]
        msg = lib.glam_last_error(pb.plan.handle)
        msg = msg.decode() if msg else ""
        if it.status not in (GLAM_OK, GLAM_ENOCONV):
            raise GlamError(it.status, f"problem {i}: {msg}")
        out.append(FitResult(list(lam), path, _stats_list(st), it.nfit, it.status, msg))
    return out
