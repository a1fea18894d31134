"""Python binding of the C ABI in include/tmop.h (argument marshalling only).

Every computation runs in libtmop_gb300.so. Tensors passed in must be
contiguous float64 CUDA tensors of shape [dim, nnode]; their data pointers go
straight to the library together with torch's current CUDA stream. If the
library is missing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtmop_gb300.so")

OK, ERR_ARG, ERR_CUDA, ERR_INVERTED, ERR_LINESEARCH, ERR_NOT_CONVERGED, ERR_CAPACITY = 0, 1, 2, 3, 4, 5, 6
GL, GLL = 0, 1
W_IDENTITY, W_CONST, W_SCALED, W_PER_QP = 0, 1, 2, 3
FP64, FP32_MIXED, FP32_BULK = 0, 1, 2
MINRES, CG = 0, 1
WT_EQUAL_SIZE, WT_LOCAL_SIZE, WT_INITIAL = 0, 1, 2


class TmopError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} (status {status})")
        self.status = status


class _Mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("nelem", C.c_int), ("nnode", C.c_int), ("elem_nodes", C.c_void_p),
                ("fixed", C.c_void_p), ("structured", C.c_int * 3)]


class _Quad(C.Structure):
    _fields_ = [("kind", C.c_int), ("npts1d", C.c_int)]


class _Targets(C.Structure):
    _fields_ = [("kind", C.c_int), ("scale", C.c_double), ("W", C.c_void_p)]


class NewtonOpts(C.Structure):
    _fields_ = [("max_newton", C.c_int), ("rtol", C.c_double), ("krylov", C.c_int), ("krylov_rtol", C.c_double),
                ("krylov_maxit", C.c_int), ("alpha_shrink", C.c_double), ("max_halvings", C.c_int),
                ("f_factor", C.c_double), ("g_factor", C.c_double), ("atol", C.c_double),
                ("matrix_free", C.c_int), ("precond", C.c_int), ("krylov_fp64", C.c_int)]


class NewtonReport(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("krylov_iterations", C.c_int),
                ("alpha", C.c_double), ("F", C.c_double), ("grad_norm", C.c_double),
                ("grad_norm0", C.c_double), ("min_detA", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

# every symbol declared in include/tmop.h, with its ctypes signature
_SIGNATURES = {
    "tmop_setup": ([C.POINTER(_Mesh), C.c_int, C.POINTER(_Quad), C.c_int, C.POINTER(_Targets), C.c_int,
                    C.POINTER(C.c_void_p)], C.c_int),
    "tmop_energy": ([C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p], C.c_int),
    "tmop_energy_device": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_gradient": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_energy_gradient": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_hess_apply": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_gradient_hess_apply": ([C.c_void_p] * 6, C.c_int),
    "tmop_newton_step": ([C.c_void_p, C.c_void_p, C.POINTER(NewtonOpts), C.POINTER(NewtonReport), C.c_void_p],
                         C.c_int),
    "tmop_newton_solve": ([C.c_void_p, C.c_void_p, C.POINTER(NewtonOpts), C.POINTER(NewtonReport), C.c_void_p],
                          C.c_int),
    "tmop_krylov_solve": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(NewtonOpts),
                           C.POINTER(C.c_int), C.c_void_p], C.c_int),
    "tmop_element_min_detA": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_linearize": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_hess_apply_pa": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_hess_apply_pa_add": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_hess_apply_pa_add_f32": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_hessian_diagonal": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_pa_layout": ([C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "tmop_sizes": ([C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)],
                   C.c_int),
    "tmop_energy_noalloc": ([C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(_Quad), C.c_int, C.POINTER(_Targets),
                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_set_composite": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_set_restricted_movement": ([C.c_void_p, C.c_double, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_jacobians": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_set_targets_from_positions": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_selftest_convert": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p], C.c_int),
    "tmop_selftest_rcbrt": ([C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p], C.c_int),
    "tmop_fma_peak": ([C.c_int, C.c_void_p, C.c_size_t, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p],
                      C.c_int),
    "tmop_precond_apply": ([C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                            C.c_void_p], C.c_int),
    "tmop_set_deterministic": ([C.c_void_p, C.c_int], C.c_int),
    "tmop_vec_add": ([C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p], C.c_int),
    "tmop_vec_axpby": ([C.c_void_p, C.c_double, C.c_void_p, C.c_double, C.c_size_t, C.c_void_p], C.c_int),
    "tmop_vec_dot_segments": ([C.c_void_p, C.c_void_p, C.c_int, C.c_size_t, C.c_size_t, C.c_size_t, C.c_void_p,
                               C.c_size_t, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_destroy": ([C.c_void_p], None),
    "tmop_status_string": ([C.c_int], C.c_char_p),
}


def load(path: str = LIB_PATH):
    """Load libtmop_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1807_09807_gb300.build.build()")
        lib = C.CDLL(path)
        for name, (args, res) in _SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def status_string(status: int) -> str:
    return load().tmop_status_string(status).decode()


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


def _check_vec(t, shape, what):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{what} must be a contiguous float64 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def selftest_convert(x):
    """(f32, back): the FP64 -> FP32 -> FP64 conversions of the FP32 kernels on x."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise TypeError("x must be a contiguous float64 CUDA tensor")
    f32 = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    back = torch.empty_like(x)
    rc = load().tmop_selftest_convert(_ptr(x), _ptr(f32), _ptr(back), x.numel(), _stream())
    if rc != OK:
        raise TmopError(rc, "tmop_selftest_convert")
    return f32, back


def selftest_rcbrt(x):
    """tau^{-1/3} as the FP64 kernels evaluate it, on x (FP64, CUDA)."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise TypeError("x must be a contiguous float64 CUDA tensor")
    out = torch.empty_like(x)
    rc = load().tmop_selftest_rcbrt(_ptr(x), _ptr(out), x.numel(), _stream())
    if rc != OK:
        raise TmopError(rc, "tmop_selftest_rcbrt")
    return out


def vec_add(y, b):
    """y += b (contiguous float64 CUDA tensors of equal size), tmop_vec_add."""
    if y.numel() != b.numel() or not (y.is_contiguous() and b.is_contiguous()):
        raise TypeError("y and b must be contiguous and of equal size")
    rc = load().tmop_vec_add(_ptr(y), _ptr(b), y.numel(), _stream())
    if rc != OK:
        raise TmopError(rc, "tmop_vec_add")


def vec_axpby(y, a, x, b):
    """y = a x + b y (contiguous float64 CUDA tensors of equal size), tmop_vec_axpby."""
    if y.numel() != x.numel() or not (y.is_contiguous() and x.is_contiguous()):
        raise TypeError("y and x must be contiguous and of equal size")
    rc = load().tmop_vec_axpby(_ptr(y), float(a), _ptr(x), float(b), y.numel(), _stream())
    if rc != OK:
        raise TmopError(rc, "tmop_vec_axpby")
    return y


def vec_dot_segments(a, b, first, count, scratch, out):
    """out (0-d float64 CUDA tensor) = sum over rows c of a[c, first:first+count] . b[...]
    for [ncomp][stride] tensors, tmop_vec_dot_segments."""
    rc = load().tmop_vec_dot_segments(_ptr(a), _ptr(b), a.shape[0], a.shape[1], first, count, _ptr(scratch),
                                      scratch.numel(), _ptr(out), _stream())
    if rc != OK:
        raise TmopError(rc, "tmop_vec_dot_segments")
    return out


PEAK_FP64, PEAK_FP32, PEAK_FP32X2 = 0, 1, 2


def fma_peak(kind=PEAK_FP64):
    """(GFLOP/s, ms): the measured FMA throughput of the current GPU
    (tmop_fma_peak), the denominator of the FP64 / FP32 ALU rooflines."""
    import torch
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    scratch = torch.empty(sms * 1024 * 8, dtype=torch.uint8, device=f"cuda:{dev}")
    g, ms = C.c_double(0.0), C.c_double(0.0)
    rc = load().tmop_fma_peak(kind, _ptr(scratch), scratch.numel(), C.byref(g), C.byref(ms), _stream())
    if rc != OK:
        raise TmopError(rc, "tmop_fma_peak")
    return g.value, ms.value


def energy_noalloc(dim, order, structured, nq, metric, x, F, min_detA, quad_kind=GL, target_kind=W_IDENTITY,
                   target_scale=1.0, W=None):
    """tmop_energy_noalloc: F and min det A of a structured grid into 0-d
    float64 CUDA tensors, with no device allocation by the library (for
    callers that must not allocate GPU memory). Returns the status code."""
    _check_vec(x, (dim, x.shape[1]), "x")
    st = (C.c_int * 3)(*(list(structured) + [0] * (3 - len(structured))))
    Wa = None if W is None else np.ascontiguousarray(W, dtype=np.float64)
    t = _Targets(target_kind, target_scale, None if Wa is None else Wa.ctypes.data)
    q = _Quad(quad_kind, nq)
    return load().tmop_energy_noalloc(dim, order, st, C.byref(q), metric, C.byref(t), _ptr(x), _ptr(F),
                                      _ptr(min_detA), _stream())


@dataclass
class NewtonResult:
    status: int
    report: dict


class Context:
    """A TMOP problem on the GPU: mesh topology, quadrature, metric, targets,
    precision form. Wraps tmop_setup / tmop_destroy."""

    def __init__(self, dim: int, order: int, nnode: int, elem_nodes: Optional[np.ndarray], fixed: Optional[np.ndarray],
                 nq: int, metric: int, quad_kind: int = GL, structured=None, target_kind: int = W_IDENTITY,
                 target_scale: float = 1.0, W: Optional[np.ndarray] = None, precision: int = FP64,
                 nelem: Optional[int] = None):
        lib = load()
        self.dim, self.order, self.nnode, self.nq, self.metric, self.precision = dim, order, nnode, nq, metric, precision
        self._en = None if elem_nodes is None else np.ascontiguousarray(elem_nodes, dtype=np.int32)
        self._fx = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8)
        self._W = None if W is None else np.ascontiguousarray(W, dtype=np.float64)
        if nelem is None:
            nelem = self._en.shape[0]
        self.nelem = nelem
        st = (C.c_int * 3)(*(list(structured) + [0] * (3 - len(structured)) if structured else [0, 0, 0]))
        m = _Mesh(dim, nelem, nnode, None if self._en is None else self._en.ctypes.data,
                  None if self._fx is None else self._fx.ctypes.data, st)
        q = _Quad(quad_kind, nq)
        t = _Targets(target_kind, target_scale, None if self._W is None else self._W.ctypes.data)
        h = C.c_void_p()
        rc = lib.tmop_setup(C.byref(m), order, C.byref(q), metric, C.byref(t), precision, C.byref(h))
        if rc != OK:
            raise TmopError(rc, "tmop_setup")
        self._h = h
        d, ne, nn, Q = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        lib.tmop_sizes(h, C.byref(d), C.byref(ne), C.byref(nn), C.byref(Q))
        self.Q = Q.value

    @classmethod
    def from_mesh(cls, m, precision: int = FP64, metric: Optional[int] = None, structured: bool = True,
                  target_scale: Optional[float] = None, W_per_qp: Optional[np.ndarray] = None):
        """Context for a meshgen.Mesh (structured fast path by default)."""
        kind, scale, W = W_IDENTITY, 1.0, None
        if W_per_qp is not None:
            kind, W = W_PER_QP, W_per_qp
        elif target_scale is not None:
            kind, scale = W_SCALED, target_scale
        elif m.W is not None:
            kind, W = W_CONST, m.W
        return cls(m.dim, m.order, m.nnode, None if structured else m.elem_nodes, m.fixed, m.nq,
                   metric or m.metric, quad_kind=m.quad_kind, structured=list(m.nx) if structured else None,
                   target_kind=kind, target_scale=scale, W=W, precision=precision, nelem=m.nelem)

    def close(self):
        if getattr(self, "_h", None):
            load().tmop_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.dim, self.nnode)

    def energy(self, x):
        """(status, F, min det A): eq. (2.4) and the det A > 0 check."""
        _check_vec(x, self.shape, "x")
        F, md = C.c_double(), C.c_double()
        rc = load().tmop_energy(self._h, _ptr(x), C.byref(F), C.byref(md), _stream())
        if rc not in (OK, ERR_INVERTED):
            raise TmopError(rc, "tmop_energy")
        return rc, F.value, md.value

    def energy_device(self, x, F, min_detA):
        """F and min det A into 0-d float64 CUDA tensors, stream ordered, no sync."""
        _check_vec(x, self.shape, "x")
        rc = load().tmop_energy_device(self._h, _ptr(x), _ptr(F), _ptr(min_detA), _stream())
        if rc != OK:
            raise TmopError(rc, "tmop_energy_device")

    def gradient(self, x, out=None):
        import torch
        _check_vec(x, self.shape, "x")
        g = torch.empty_like(x) if out is None else out
        _check_vec(g, self.shape, "g")
        rc = load().tmop_gradient(self._h, _ptr(x), _ptr(g), _stream())
        if rc != OK:
            raise TmopError(rc, "tmop_gradient")
        return g

    def energy_gradient(self, x, out=None):
        """(g, F, min det A) of x: g = dF/dx into `out` and F, min det A as
        0-d device tensors, in one element pass where the context allows it."""
        import torch
        _check_vec(x, self.shape, "x")
        g = torch.empty_like(x) if out is None else out
        _check_vec(g, self.shape, "g")
        fm = torch.empty(2, dtype=torch.float64, device=x.device)
        rc = load().tmop_energy_gradient(self._h, _ptr(x), _ptr(g), fm.data_ptr(), fm.data_ptr() + 8, _stream())
        if rc != OK:
            raise TmopError(rc, "tmop_energy_gradient")
        return g, fm[0], fm[1]

    def hess_apply(self, x, v, out=None):
        import torch
        _check_vec(x, self.shape, "x")
        _check_vec(v, self.shape, "v")
        y = torch.empty_like(x) if out is None else out
        _check_vec(y, self.shape, "y")
        rc = load().tmop_hess_apply(self._h, _ptr(x), _ptr(v), _ptr(y), _stream())
        if rc != OK:
            raise TmopError(rc, "tmop_hess_apply")
        return y

    def gradient_hess_apply(self, x, v, g=None, y=None):
        """(g, y) = (dF/dx, H(x) v) at the same x, in one element pass where
        the context allows (tmop_gradient_hess_apply)."""
        import torch
        _check_vec(x, self.shape, "x")
        _check_vec(v, self.shape, "v")
        g = torch.empty_like(x) if g is None else g
        y = torch.empty_like(x) if y is None else y
        _check_vec(g, self.shape, "g")
        _check_vec(y, self.shape, "y")
        rc = load().tmop_gradient_hess_apply(self._h, _ptr(x), _ptr(v), _ptr(g), _ptr(y), _stream())
        if rc != OK:
            raise TmopError(rc, "tmop_gradient_hess_apply")
        return g, y

    def set_composite(self, metric2: int, W2=None, eta2=None):
        """Second metric term eta_q mu2(A W2^-1) (eq. (4.1)); metric2 = 0 removes it."""
        W2a = None if W2 is None else np.ascontiguousarray(W2, dtype=np.float64)
        eta = None if eta2 is None else np.ascontiguousarray(eta2, dtype=np.float64)
        if metric2 and W2a is None:
            W2a = np.eye(self.dim)
        rc = load().tmop_set_composite(self._h, metric2, None if W2a is None else W2a.ctypes.data,
                                       None if eta is None else eta.ctypes.data)
        if rc != OK:
            raise TmopError(rc, "tmop_set_composite")

    def set_restricted_movement(self, delta: float, x_init=None):
        """Add delta |x - x_init|^2 integrated over the target elements (eq. (4.2))."""
        if x_init is not None:
            _check_vec(x_init, self.shape, "x_init")
        rc = load().tmop_set_restricted_movement(self._h, float(delta), None if x_init is None else _ptr(x_init),
                                                 _stream())
        if rc != OK:
            raise TmopError(rc, "tmop_set_restricted_movement")

    def jacobians(self, x, out=None):
        """A(x) at every quadrature point, [nelem, Q, dim, dim] (eq. (2.2))."""
        import torch
        _check_vec(x, self.shape, "x")
        J = torch.empty((self.nelem, self.Q, self.dim, self.dim), dtype=torch.float64, device=x.device) \
            if out is None else out
        if not (J.is_cuda and J.dtype == torch.float64 and J.is_contiguous()
                and tuple(J.shape) == (self.nelem, self.Q, self.dim, self.dim)):
            raise ValueError("out must be a contiguous float64 CUDA tensor [nelem, Q, dim, dim]")
        rc = load().tmop_jacobians(self._h, _ptr(x), _ptr(J), _stream())
        if rc != OK:
            raise TmopError(rc, "tmop_jacobians")
        return J

    def set_targets_from_positions(self, kind: int, x0):
        """Targets built from positions x0: WT_EQUAL_SIZE (W2, eq. (3.1)),
        WT_LOCAL_SIZE (W3, Section 3.1) or WT_INITIAL (W0 = A(x0), Section 4.3.2)."""
        _check_vec(x0, self.shape, "x0")
        rc = load().tmop_set_targets_from_positions(self._h, int(kind), _ptr(x0), _stream())
        if rc != OK:
            raise TmopError(rc, "tmop_set_targets_from_positions")

    def linearize(self, x):
        """Store the per-point Hessians at x (partial assembly)."""
        _check_vec(x, self.shape, "x")
        rc = load().tmop_linearize(self._h, _ptr(x), _stream())
        if rc != OK:
            raise TmopError(rc, "tmop_linearize")

    def hess_apply_pa(self, v, out=None, accumulate=False):
        """y = H v with the Hessians of the last linearize(); accumulate: y += H v
        into `out` (tmop_hess_apply_pa_add: y is not zeroed first)."""
        import torch
        _check_vec(v, self.shape, "v")
        if accumulate and out is None:
            raise ValueError("accumulate needs out")
        y = torch.empty_like(v) if out is None else out
        _check_vec(y, self.shape, "y")
        fn = "tmop_hess_apply_pa_add" if accumulate else "tmop_hess_apply_pa"
        rc = getattr(load(), fn)(self._h, _ptr(v), _ptr(y), _stream())
        if rc != OK:
            raise TmopError(rc, fn)
        return y

    def hess_apply_pa_add_f32(self, v, y):
        """y += H v on FP32 vectors (tmop_hess_apply_pa_add_f32; FP32 contexts)."""
        import torch
        for t, nm in ((v, "v"), (y, "y")):
            if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != tuple(self.shape):
                raise ValueError(f"{nm} must be a contiguous CUDA float32 tensor of shape {self.shape}")
        rc = load().tmop_hess_apply_pa_add_f32(self._h, _ptr(v), _ptr(y), _stream())
        if rc != OK:
            raise TmopError(rc, "tmop_hess_apply_pa_add_f32")
        return y

    def pa_layout(self):
        """(values per point, element stride, bytes per value) of the stored linearisation."""
        v, st, b = C.c_int(0), C.c_int(0), C.c_int(0)
        rc = load().tmop_pa_layout(self._h, C.byref(v), C.byref(st), C.byref(b))
        if rc != OK:
            raise TmopError(rc, "tmop_pa_layout")
        return v.value, st.value, b.value

    def hessian_diagonal(self, out=None):
        """Diagonal of the Hessian stored by the last linearize() (1 at fixed dofs)."""
        import torch
        d = torch.empty(self.shape, dtype=torch.float64, device="cuda") if out is None else out
        _check_vec(d, self.shape, "out")
        rc = load().tmop_hessian_diagonal(self._h, _ptr(d), _stream())
        if rc != OK:
            raise TmopError(rc, "tmop_hessian_diagonal")
        return d

    def element_min_detA(self, x, out=None):
        import torch
        _check_vec(x, self.shape, "x")
        o = torch.empty(self.nelem, dtype=torch.float64, device=x.device) if out is None else out
        rc = load().tmop_element_min_detA(self._h, _ptr(x), _ptr(o), _stream())
        if rc != OK:
            raise TmopError(rc, "tmop_element_min_detA")
        return o

    @staticmethod
    def opts(**kw) -> NewtonOpts:
        o = NewtonOpts()
        for k, v in kw.items():
            if k == "krylov" and isinstance(v, str):
                v = CG if v == "cg" else MINRES
            setattr(o, k, v)
        return o

    def set_deterministic(self, on=True):
        """Colour-ordered nodal sums (bitwise reproducible) instead of atomics."""
        rc = load().tmop_set_deterministic(self._h, 1 if on else 0)
        if rc != OK:
            raise TmopError(rc, "tmop_set_deterministic")

    def precond_apply(self, x, r, precond=2):
        """(z, alpha): z = M^-1 r for the linearisation at x (tmop_precond_apply)."""
        import torch
        _check_vec(x, self.shape, "x")
        _check_vec(r, self.shape, "r")
        z = torch.empty_like(r)
        a = C.c_double(0.0)
        rc = load().tmop_precond_apply(self._h, _ptr(x), int(precond), _ptr(r), _ptr(z), C.byref(a), _stream())
        if rc != OK:
            raise TmopError(rc, "tmop_precond_apply")
        return z, a.value

    def krylov_solve(self, x, b, out=None, **kw):
        import torch
        _check_vec(x, self.shape, "x")
        _check_vec(b, self.shape, "b")
        p = torch.empty_like(x) if out is None else out
        it = C.c_int()
        o = self.opts(**kw)
        rc = load().tmop_krylov_solve(self._h, _ptr(x), _ptr(b), _ptr(p), C.byref(o), C.byref(it), _stream())
        if rc != OK:
            raise TmopError(rc, "tmop_krylov_solve")
        return p, it.value

    def newton_step(self, x, **kw) -> NewtonResult:
        _check_vec(x, self.shape, "x")
        o, r = self.opts(**kw), NewtonReport()
        rc = load().tmop_newton_step(self._h, _ptr(x), C.byref(o), C.byref(r), _stream())
        if rc in (ERR_ARG, ERR_CUDA):
            raise TmopError(rc, "tmop_newton_step")
        return NewtonResult(rc, r.as_dict())

    def newton_solve(self, x, **kw) -> NewtonResult:
        _check_vec(x, self.shape, "x")
        o, r = self.opts(**kw), NewtonReport()
        rc = load().tmop_newton_solve(self._h, _ptr(x), C.byref(o), C.byref(r), _stream())
        if rc in (ERR_ARG, ERR_CUDA):
            raise TmopError(rc, "tmop_newton_solve")
        return NewtonResult(rc, r.as_dict())
