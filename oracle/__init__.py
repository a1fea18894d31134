"""Plain FP64 CPU oracle for high-order TMOP (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package. The GPU library never does: it shares no code
with ``tmop_oracle.c``. The C source is compiled with gcc on first use (or by
``build()``) into ``oracle/_build/liboracle.so``.

Every function follows the paper's formulas directly:
  * ``energy``      -- eq. (2.4), F_V = sum_E sum_q w_q det W mu(T), T = A W^-1
  * ``gradient``    -- Section 3.4, dF_V/dx_i = sum_E int (grad phi_i W^-1) : dmu/dT
  * ``hess_apply``  -- Section 3.4, the Hessian from second derivatives of mu
  * ``metric``      -- Table 3.1 and Section 3.2 metrics with P and dP
  * ``newton``      -- Section 3.4 damped Newton with the det(A) > 0, 1.2 F and
                       1.2 |g| line-search rules, MINRES inner solves (Section 5)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tmop_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_INVERTED, ERR_LINESEARCH, ERR_NOT_CONVERGED = 0, 1, 3, 4, 5
GL, GLL = 0, 1
W_IDENTITY, W_CONST, W_PER_QP = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, -O2, no vectorisation flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Problem(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("order", C.c_int), ("nelem", C.c_int), ("nnode", C.c_int),
        ("elem_nodes", C.c_void_p), ("fixed", C.c_void_p),
        ("quad_kind", C.c_int), ("nq", C.c_int), ("metric", C.c_int),
        ("wkind", C.c_int), ("W", C.c_void_p),
        ("metric2", C.c_int), ("W2", C.c_void_p), ("eta2", C.c_void_p),
        ("delta", C.c_double), ("x_init", C.c_void_p),
    ]


class _NewtonOpts(C.Structure):
    _fields_ = [
        ("max_newton", C.c_int), ("rtol", C.c_double), ("krylov", C.c_int),
        ("krylov_rtol", C.c_double), ("krylov_maxit", C.c_int), ("alpha_shrink", C.c_double),
        ("max_halvings", C.c_int), ("f_factor", C.c_double), ("g_factor", C.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER(_Problem)
            dp, ip = C.c_void_p, C.c_void_p
            lib.orc_gauss_legendre.argtypes = [C.c_int, dp, dp]
            lib.orc_gauss_lobatto.argtypes = [C.c_int, dp, dp]
            lib.orc_lagrange.argtypes = [C.c_int, dp, C.c_double, dp, dp]
            lib.orc_lagrange.restype = None
            lib.orc_metric.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp, dp]
            lib.orc_jacobians.argtypes = [P, dp, dp]
            lib.orc_tables_dump.argtypes = [P, dp, dp]
            lib.orc_energy.argtypes = [P, dp, ip, C.c_int, dp, dp]
            lib.orc_gradient.argtypes = [P, dp, ip, C.c_int, dp]
            lib.orc_hess_apply.argtypes = [P, dp, dp, ip, C.c_int, dp]
            lib.orc_minres.argtypes = [P, dp, dp, C.c_double, C.c_int, dp]
            lib.orc_cg.argtypes = [P, dp, dp, C.c_double, C.c_int, dp]
            lib.orc_newton.argtypes = [P, dp, C.POINTER(_NewtonOpts), dp, C.POINTER(C.c_int)]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def gauss_legendre(q: int):
    pts, wts = np.zeros(q), np.zeros(q)
    if _load().orc_gauss_legendre(q, _ptr(pts), _ptr(wts)) != OK:
        raise ValueError("bad q")
    return pts, wts


def gauss_lobatto(q: int):
    pts, wts = np.zeros(q), np.zeros(q)
    if _load().orc_gauss_lobatto(q, _ptr(pts), _ptr(wts)) != OK:
        raise ValueError("bad q")
    return pts, wts


def lagrange(nodes, xi: float):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    n = len(nodes)
    phi, dphi = np.zeros(n), np.zeros(n)
    _load().orc_lagrange(n, _ptr(nodes), float(xi), _ptr(phi), _ptr(dphi))
    return phi, dphi


def metric(mid: int, T, dT=None):
    """mu(T), P = dmu/dT and (if dT is given) dP = d^2mu/dT^2 : dT. Returns
    (status, mu, P, dP)."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    d = T.shape[0]
    mu = np.zeros(1)
    P = np.zeros((d, d))
    dP = None if dT is None else np.zeros((d, d))
    dTa = None if dT is None else np.ascontiguousarray(dT, dtype=np.float64)
    rc = _load().orc_metric(mid, d, _ptr(T), _ptr(dTa), _ptr(mu), _ptr(P), _ptr(dP))
    return rc, float(mu[0]), P, dP


@dataclass
class Problem:
    """A TMOP problem as the oracle sees it (host arrays)."""
    dim: int
    order: int
    elem_nodes: np.ndarray      # int32 [nelem, (order+1)^dim]
    nnode: int
    fixed: np.ndarray | None    # uint8 [dim, nnode]
    nq: int
    metric: int
    quad_kind: int = GL
    wkind: int = W_IDENTITY
    W: np.ndarray | None = None  # [d,d] (W_CONST) or [nelem, Q, d, d] (W_PER_QP)
    metric2: int = 0             # composite second term (eq. (4.1)); 0 = none
    W2: np.ndarray | None = None  # [d,d] constant target of the second term
    eta2: np.ndarray | None = None  # [nelem, Q] weights of the second term (None = 1)
    delta: float = 0.0           # restricted movement weight (eq. (4.2)); 0 = none
    x_init: np.ndarray | None = None  # [dim, nnode] reference positions of that term

    def __post_init__(self):
        self.elem_nodes = np.ascontiguousarray(self.elem_nodes, dtype=np.int32)
        if self.fixed is not None:
            self.fixed = np.ascontiguousarray(self.fixed, dtype=np.uint8)
        if self.W is not None:
            self.W = np.ascontiguousarray(self.W, dtype=np.float64)
        if self.metric2:
            self.W2 = np.ascontiguousarray(np.eye(self.dim) if self.W2 is None else self.W2, dtype=np.float64)
        if self.eta2 is not None:
            self.eta2 = np.ascontiguousarray(self.eta2, dtype=np.float64)
        if self.delta:
            self.x_init = np.ascontiguousarray(self.x_init, dtype=np.float64)
        self._c = _Problem(self.dim, self.order, self.elem_nodes.shape[0], self.nnode,
                           _ptr(self.elem_nodes), _ptr(self.fixed), self.quad_kind, self.nq,
                           self.metric, self.wkind, _ptr(self.W), self.metric2, _ptr(self.W2), _ptr(self.eta2),
                           float(self.delta), _ptr(self.x_init))

    @property
    def nelem(self):
        return self.elem_nodes.shape[0]

    @property
    def Q(self):
        return self.nq ** self.dim

    def _x(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        assert x.shape == (self.dim, self.nnode), x.shape
        return x

    @staticmethod
    def _elems(elems):
        if elems is None:
            return None, 0
        e = np.ascontiguousarray(elems, dtype=np.int32)
        return e, len(e)

    def energy(self, x, elems=None):
        """(status, F, min det A) -- eq. (2.4)."""
        x = self._x(x)
        e, ne = self._elems(elems)
        F, md = np.zeros(1), np.zeros(1)
        rc = _load().orc_energy(C.byref(self._c), _ptr(x), _ptr(e), ne, _ptr(F), _ptr(md))
        if rc == ERR_ARG:
            raise ValueError("oracle energy: bad argument")
        return rc, float(F[0]), float(md[0])

    def gradient(self, x, elems=None):
        x = self._x(x)
        e, ne = self._elems(elems)
        g = np.zeros_like(x)
        rc = _load().orc_gradient(C.byref(self._c), _ptr(x), _ptr(e), ne, _ptr(g))
        if rc == ERR_ARG:
            raise ValueError("oracle gradient: bad argument")
        return g

    def hess_apply(self, x, v, elems=None):
        x = self._x(x)
        v = self._x(v)
        e, ne = self._elems(elems)
        y = np.zeros_like(x)
        rc = _load().orc_hess_apply(C.byref(self._c), _ptr(x), _ptr(v), _ptr(e), ne, _ptr(y))
        if rc == ERR_ARG:
            raise ValueError("oracle hess_apply: bad argument")
        return y

    def jacobians(self, x):
        x = self._x(x)
        out = np.zeros((self.nelem, self.Q, self.dim, self.dim))
        if _load().orc_jacobians(C.byref(self._c), _ptr(x), _ptr(out)) != OK:
            raise ValueError("bad problem")
        return out

    def tables(self):
        """(w [Q], gradphi [Q, n^d, d]) as the oracle uses them."""
        nd = (self.order + 1) ** self.dim
        w = np.zeros(self.Q)
        gp = np.zeros((self.Q, nd, self.dim))
        if _load().orc_tables_dump(C.byref(self._c), _ptr(w), _ptr(gp)) != OK:
            raise ValueError("bad problem")
        return w, gp

    def minres(self, x, b, rtol=1e-10, maxit=2000):
        x, b = self._x(x), self._x(b)
        s = np.zeros_like(x)
        it = _load().orc_minres(C.byref(self._c), _ptr(x), _ptr(b), rtol, maxit, _ptr(s))
        return s, it

    def cg(self, x, b, rtol=1e-10, maxit=2000):
        x, b = self._x(x), self._x(b)
        s = np.zeros_like(x)
        it = _load().orc_cg(C.byref(self._c), _ptr(x), _ptr(b), rtol, maxit, _ptr(s))
        return s, it

    def newton(self, x, max_newton=10, rtol=1e-12, krylov="minres", krylov_rtol=1e-10,
               krylov_maxit=2000, alpha_shrink=0.5, max_halvings=30, f_factor=1.2, g_factor=1.2):
        """Section 3.4 Newton. Returns (status, x_final, history[iters+1, 5]) with
        history columns F, |g|, min det A, alpha, Krylov iterations."""
        x = self._x(x).copy()
        o = _NewtonOpts(max_newton, rtol, 1 if krylov == "cg" else 0, krylov_rtol, krylov_maxit,
                        alpha_shrink, max_halvings, f_factor, g_factor)
        hist = np.zeros((max_newton + 1, 5))
        its = C.c_int(0)
        rc = _load().orc_newton(C.byref(self._c), _ptr(x), C.byref(o), _ptr(hist), C.byref(its))
        return rc, x, hist[: its.value + 1]
