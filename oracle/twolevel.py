"""Plain dense reference of the two-level Krylov preconditioner (test
infrastructure only; nothing in the GPU library imports it).

Section 5 runs MINRES on the Newton system; the paper does not state its
preconditioner. The library's two-level choice, written here from its
definition with dense numpy matrices, no transforms and no tensor tricks:

    M^-1 r = D^-1 r + P (alpha K_c)^-1 P^t r

* P: the vertex field of each element (bilinear in 2D, trilinear in 3D, on
  the reference element [0,1]^d) evaluated at the element's order-k
  Gauss-Lobatto lattice nodes; interior vertices only (the boundary is
  fixed). Built entry by entry from the 1D hat functions.
* K_c: the reference-space Q1 Laplacian of the vertex field,
  sum_E int grad N_a . grad N_b over the unit reference element, assembled
  element by element from the exact Q1 element matrix, interior vertices.
* alpha = (P w)^t H (P w) / (w^t K_c w) for w the eigenvector of K_c with
  the smallest eigenvalue, placed in every component.
* D^-1: the inverse Hessian diagonal, passed in by the caller.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import gauss_lobatto


def hat_interpolation(n: int, k: int) -> np.ndarray:
    """[k n + 1][n - 1]: 1D lattice node g = k e + i (GLL node z_i of element e)
    takes (1 - z_i) of vertex e and z_i of vertex e + 1; columns are the
    interior vertices 1..n-1."""
    z, _ = gauss_lobatto(k + 1)
    P = np.zeros((k * n + 1, n + 1))
    for e in range(n):
        for i in range(k + 1):
            g = k * e + i
            P[g, e] = 1.0 - z[i]
            P[g, e + 1] = z[i]
    return P[:, 1:-1]


def interpolation(ns, k: int) -> np.ndarray:
    """Scalar P for a grid of ns = (nx, ny[, nz]) elements: lattice node
    (x fastest) from interior vertex (x fastest), the product of the 1D hats."""
    P1 = [hat_interpolation(n, k) for n in ns]
    Lf = [k * n + 1 for n in ns]
    Lc = [n - 1 for n in ns]
    P = np.zeros((int(np.prod(Lf)), int(np.prod(Lc))))
    for gf in itertools.product(*[range(L) for L in reversed(Lf)]):
        gf = gf[::-1]                                    # (gx, gy[, gz])
        row = 0
        for a in reversed(range(len(ns))):
            row = row * Lf[a] + gf[a]
        for vc in itertools.product(*[range(L) for L in reversed(Lc)]):
            vc = vc[::-1]
            w = 1.0
            for a in range(len(ns)):
                w *= P1[a][gf[a], vc[a]]
            if w != 0.0:
                col = 0
                for a in reversed(range(len(ns))):
                    col = col * Lc[a] + vc[a]
                P[row, col] = w
    return P


def q1_element_stiffness(dim: int) -> np.ndarray:
    """int over [0,1]^d of grad N_a . grad N_b for the 2^d vertex functions
    (vertex index a = sum_b bit_b(a) 2^b, x fastest), from the exact 1D
    integrals: int N0 N0 = 1/3, int N0 N1 = 1/6, int N0' N0' = 1, N0' N1' = -1."""
    m1 = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    k1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    nv = 2 ** dim
    K = np.zeros((nv, nv))
    for a in range(nv):
        for b in range(nv):
            s = 0.0
            for axis in range(dim):
                t = 1.0
                for c in range(dim):
                    ia, ib = (a >> c) & 1, (b >> c) & 1
                    t *= k1[ia, ib] if c == axis else m1[ia, ib]
                s += t
            K[a, b] = s
    return K


def coarse_laplacian(ns) -> np.ndarray:
    """Assembled Q1 reference-space Laplacian on the interior vertices."""
    dim = len(ns)
    V = [n + 1 for n in ns]
    Ke = q1_element_stiffness(dim)
    N = int(np.prod(V))
    K = np.zeros((N, N))
    for e in itertools.product(*[range(n) for n in reversed(ns)]):
        e = e[::-1]
        ids = []
        for a in range(2 ** dim):
            v = [e[c] + ((a >> c) & 1) for c in range(dim)]
            idx = 0
            for c in reversed(range(dim)):
                idx = idx * V[c] + v[c]
            ids.append(idx)
        K[np.ix_(ids, ids)] += Ke
    interior = []
    for v in itertools.product(*[range(n) for n in reversed(V)]):
        v = v[::-1]
        if all(0 < v[c] < V[c] - 1 for c in range(dim)):
            idx = 0
            for c in reversed(range(dim)):
                idx = idx * V[c] + v[c]
            interior.append(idx)
    return K[np.ix_(interior, interior)]


def alpha(hess_apply, ns, k: int, dim: int) -> float:
    """Rayleigh quotient (P w)^t H (P w) / (w^t K_c w), w the smoothest
    eigenvector of K_c in every component; hess_apply maps a [dim][N] array
    to H times it."""
    P = interpolation(ns, k)
    Kc = coarse_laplacian(ns)
    lam, vec = np.linalg.eigh(Kc)
    w0 = vec[:, 0]
    Pw = np.stack([P @ w0] * dim)
    Hw = hess_apply(Pw)
    return float(np.sum(Pw * Hw) / (dim * w0 @ Kc @ w0))


def coarse_part(r: np.ndarray, ns, k: int, a: float) -> np.ndarray:
    """P (a K_c)^-1 P^t r per component, r [dim][N]."""
    P = interpolation(ns, k)
    Kc = coarse_laplacian(ns)
    return np.stack([P @ np.linalg.solve(a * Kc, P.T @ rc) for rc in r])


def apply(r: np.ndarray, dinv: np.ndarray, ns, k: int, a: float) -> np.ndarray:
    """M^-1 r = D^-1 r + P (a K_c)^-1 P^t r."""
    return dinv * r + coarse_part(r, ns, k, a)
