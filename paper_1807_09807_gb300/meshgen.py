"""Seeded synthetic TMOP inputs: structured quad/hex meshes of order k with
perturbed interior nodes, shaped like the paper's 2D/3D test meshes
(Section 5: order 2-4 quads and hexes, interior nodes displaced, boundary
fixed). The paper's own meshes (turbine blade, ICF, pinched sphere) are not
available, so these stand in for them.

This module holds the inputs only: node placement, connectivity, the fixed
boundary mask and the random perturbations. It contains none of the method's
arithmetic (no basis, quadrature, Jacobian or metric); both the GPU library's
callers and the CPU oracle take their inputs from here.

Layout conventions:
  * reference element [0,1]^d, nodal Lagrange basis on Gauss-Lobatto points;
  * global nodes of an (nx, ny[, nz]) grid of order k form a lexicographic
    (k*nx+1) x (k*ny+1) [x (k*nz+1)] lattice, x fastest;
  * element e = (ex, ey[, ez]) with ex fastest; its local nodes are numbered
    lexicographically with x fastest;
  * positions are SoA float64 [d][nnode].

Random numbers: splitmix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", 2014), counter form z_n = mix(seed +
(n+1) * 0x9E3779B97F4A7C15), n = node * d + component, mapped to U(-1, 1) by
((z >> 11) * 2^-53) * 2 - 1.
"""
from __future__ import annotations

from dataclasses import dataclass, replace
from typing import Callable, Optional

import numpy as np

# Gauss-Lobatto node positions on [0,1] for orders 1..4 (closed forms: the
# interior points are the roots of P'_k, e.g. +-1/sqrt(5) for k = 3).
_GLL_NODES = {
    1: (0.0, 1.0),
    2: (0.0, 0.5, 1.0),
    3: (0.0, 0.5 * (1.0 - 1.0 / np.sqrt(5.0)), 0.5 * (1.0 + 1.0 / np.sqrt(5.0)), 1.0),
    4: (0.0, 0.5 * (1.0 - np.sqrt(3.0 / 7.0)), 0.5, 0.5 * (1.0 + np.sqrt(3.0 / 7.0)), 1.0),
}

GL, GLL = 0, 1
W_IDENTITY, W_CONST, W_PER_QP = 0, 1, 2

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of the splitmix64 stream seeded by seed."""
    with np.errstate(over="ignore"):
        n = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + n * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """U(-1, 1) doubles from splitmix64: ((z >> 11) * 2^-53) * 2 - 1."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


@dataclass
class Mesh:
    """A structured order-k quad/hex mesh and the TMOP problem set on it."""
    dim: int
    order: int
    nx: tuple                 # elements per axis
    x: np.ndarray             # float64 [d][nnode], perturbed positions
    x_ideal: np.ndarray       # float64 [d][nnode], before the random jitter
    elem_nodes: np.ndarray    # int32 [nelem][(k+1)^d]
    fixed: np.ndarray         # uint8 [d][nnode]
    nq: int = 4               # quadrature points per direction
    quad_kind: int = GL
    metric: int = 2
    wkind: int = W_IDENTITY
    W: Optional[np.ndarray] = None   # [d][d] for W_CONST
    seed: int = 1
    attempts: int = 1
    name: str = ""

    @property
    def nnode(self) -> int:
        return self.x.shape[1]

    @property
    def nelem(self) -> int:
        return self.elem_nodes.shape[0]

    @property
    def nodes_per_axis(self) -> tuple:
        return tuple(self.order * n + 1 for n in self.nx)

    @property
    def Q(self) -> int:
        return self.nq ** self.dim

    @property
    def n_qp(self) -> int:
        return self.nelem * self.Q


def lattice_coordinates(order: int, nx: int) -> np.ndarray:
    """1D coordinates of the k*nx+1 global nodes of a uniform [0,1] grid with
    Gauss-Lobatto node placement inside each element."""
    xi = np.array(_GLL_NODES[order])
    g = np.arange(order * nx + 1)
    e = np.minimum(g // order, nx - 1)
    i = g - e * order
    return (e + xi[i]) / nx


def structured(dim: int, order: int, nx) -> tuple:
    """Uniform grid on [0,1]^d: (x [d][nnode], elem_nodes, fixed boundary mask)."""
    nx = tuple(int(v) for v in (nx if np.ndim(nx) else (nx,) * dim))
    assert len(nx) == dim and order in _GLL_NODES
    n = order + 1
    Nax = [order * v + 1 for v in nx]
    axes = [lattice_coordinates(order, v) for v in nx]
    if dim == 2:
        Y, X = np.meshgrid(axes[1], axes[0], indexing="ij")
        x = np.stack([X.ravel(), Y.ravel()])
        idx = np.arange(Nax[0] * Nax[1]).reshape(Nax[1], Nax[0])
        ey, ex = np.meshgrid(np.arange(nx[1]), np.arange(nx[0]), indexing="ij")
        lj, li = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        rows = ey.ravel()[:, None] * order + lj.ravel()[None, :]
        cols = ex.ravel()[:, None] * order + li.ravel()[None, :]
        elem_nodes = idx[rows, cols]
        jj, ii = np.meshgrid(np.arange(Nax[1]), np.arange(Nax[0]), indexing="ij")
        bnd = (ii == 0) | (ii == Nax[0] - 1) | (jj == 0) | (jj == Nax[1] - 1)
    else:
        Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
        x = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
        idx = np.arange(Nax[0] * Nax[1] * Nax[2]).reshape(Nax[2], Nax[1], Nax[0])
        ez, ey, ex = np.meshgrid(np.arange(nx[2]), np.arange(nx[1]), np.arange(nx[0]), indexing="ij")
        ll, lj, li = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        pl = ez.ravel()[:, None] * order + ll.ravel()[None, :]
        rows = ey.ravel()[:, None] * order + lj.ravel()[None, :]
        cols = ex.ravel()[:, None] * order + li.ravel()[None, :]
        elem_nodes = idx[pl, rows, cols]
        kk, jj, ii = np.meshgrid(np.arange(Nax[2]), np.arange(Nax[1]), np.arange(Nax[0]), indexing="ij")
        bnd = ((ii == 0) | (ii == Nax[0] - 1) | (jj == 0) | (jj == Nax[1] - 1) |
               (kk == 0) | (kk == Nax[2] - 1))
    fixed = np.repeat(bnd.ravel()[None, :], dim, axis=0).astype(np.uint8)
    return np.ascontiguousarray(x), np.ascontiguousarray(elem_nodes.astype(np.int32)), fixed


def tangential_mask(x_lattice_shape: tuple, dim: int) -> np.ndarray:
    """Fixed-dof mask for boundary nodes that may slide along the axis-parallel
    faces of the unit square/cube (Section 4.1: boundary motion allowed only
    on boundaries parallel to the coordinate axes, imposed as Dirichlet
    conditions on the displacement): component c of a node is fixed iff the
    node lies on a face normal to axis c. Corners and edges therefore fix
    every component normal to one of their faces."""
    Nax = x_lattice_shape
    idx = np.indices(tuple(reversed(Nax)))          # (z,) y, x index grids
    comp = list(reversed([i.ravel() for i in idx]))  # x index first
    fixed = np.zeros((dim, int(np.prod(Nax))), dtype=np.uint8)
    for c in range(dim):
        fixed[c] = ((comp[c] == 0) | (comp[c] == Nax[c] - 1)).astype(np.uint8)
    return fixed


def jitter(x: np.ndarray, fixed: np.ndarray, amplitude: float, seed: int) -> np.ndarray:
    """Add U(-amplitude, amplitude) to every free coordinate. The draw index is
    node * d + component (node-major), drawn for every node."""
    d, N = x.shape
    u = uniform_pm1(seed, d * N).reshape(N, d).T
    return x + amplitude * u * (1 - fixed)


def shear(x: np.ndarray) -> np.ndarray:
    """Trilinear shear (x, y, z) -> (x + 0.2 y + 0.1 y z, y + 0.1 z, z). Its
    Jacobian has determinant 1, and it is bilinear on every face, so an order
    k >= 1 mesh represents it exactly."""
    X, Y, Z = x
    return np.stack([X + 0.2 * Y + 0.1 * Y * Z, Y + 0.1 * Z, Z])


# Workloads shaped like the paper's tests (Section 5): (dim, order, elements per
# axis, 1D quadrature points, jitter in units of the node spacing h, extra
# deformation, metric).
PRESETS = {
    # 2D order 2, 8x8 quads, 4x4 Gauss points, mu2, W = I, jitter +-0.15h
    "c1": dict(dim=2, order=2, nx=8, nq=4, jitter=0.15, deform=None, metric=2),
    # 2D order 3, 64x64 quads, x += 0.05 sin(2 pi x) sin(2 pi y), jitter +-0.1h, 5x5 points
    "c2": dict(dim=2, order=3, nx=64, nq=5, jitter=0.10, deform="sine", metric=2),
    # 3D order 2, 32^3 hexes, jitter +-0.1h then trilinear shear, 4x4x4 points
    "c3": dict(dim=3, order=2, nx=32, nq=4, jitter=0.10, deform="shear", metric=303),
    # 3D order 3, 48^3 hexes, same deformation, 5x5x5 points, mu303
    "c4": dict(dim=3, order=3, nx=48, nq=5, jitter=0.10, deform="shear", metric=303),
    # learned-proposal meshes: 2D order 3, jitter +-0.15h, mu2 (32x32 train, 128x128 apply)
    "c5": dict(dim=2, order=3, nx=32, nq=5, jitter=0.15, deform=None, metric=2),
    "c5apply": dict(dim=2, order=3, nx=128, nq=5, jitter=0.15, deform=None, metric=2),
    # the same with a curved top boundary y = 1 + 0.15 sin(pi x) (all boundary
    # nodes fixed on it): the minimiser is no longer the uniform grid
    "c5curved": dict(dim=2, order=3, nx=32, nq=5, jitter=0.15, deform="bump", metric=2),
    "c5curvedapply": dict(dim=2, order=3, nx=128, nq=5, jitter=0.15, deform="bump", metric=2),
}

REDRAW_STRIDE = 1_000_003
MAX_ATTEMPTS = 100


def make_mesh(name: str = "c1", seed: int = 1, accept: Optional[Callable[["Mesh"], bool]] = None,
              **overrides) -> Mesh:
    """Build a preset workload. If ``accept`` is given (a caller-supplied
    validity check, e.g. "every det A > 0"), the jitter is redrawn with seed
    seed + attempt * 1_000_003 until it accepts, up to 100 attempts."""
    cfg = dict(PRESETS[name])
    cfg.update(overrides)
    dim, order, nx = cfg["dim"], cfg["order"], cfg["nx"]
    x0, en, fixed = structured(dim, order, nx)
    nxt = tuple(nx if np.ndim(nx) else (nx,) * dim)
    if cfg.get("tangential"):
        # boundary nodes keep their normal coordinate and slide along the face
        fixed = tangential_mask(tuple(order * v + 1 for v in nxt), dim)
    if cfg.get("deform") == "sine" and dim == 2:
        # only the x-component; sin(2 pi x) sin(2 pi y) vanishes on the boundary
        x0 = x0.copy()
        x0[0] += 0.05 * np.sin(2 * np.pi * x0[0]) * np.sin(2 * np.pi * x0[1])
    if cfg.get("deform") == "bump" and dim == 2:
        # y -> y (1 + a sin(pi x)): the top edge becomes the curve 1 + a sin(pi x)
        x0 = x0.copy()
        x0[1] *= 1.0 + float(cfg.get("bump", 0.15)) * np.sin(np.pi * x0[0])
    # h is the node spacing of the order-k lattice, 1 / (k * n_x): jitter is
    # measured against the distance between neighbouring nodes.
    h = 1.0 / (order * max(nxt))
    wkind, W = W_IDENTITY, None
    if cfg.get("target_scale") is not None:
        wkind, W = W_CONST, np.eye(dim) * float(cfg["target_scale"])
    for attempt in range(MAX_ATTEMPTS):
        s = seed + attempt * REDRAW_STRIDE
        x = jitter(x0, fixed, cfg["jitter"] * h, s)
        xi = x0
        if cfg.get("deform") == "shear" and dim == 3:
            x, xi = shear(x), shear(x0)
        m = Mesh(dim=dim, order=order, nx=nxt, x=np.ascontiguousarray(x), x_ideal=np.ascontiguousarray(xi),
                 elem_nodes=en, fixed=fixed, nq=cfg["nq"], quad_kind=cfg.get("quad_kind", GL),
                 metric=cfg["metric"], wkind=wkind, W=W, seed=s, attempts=attempt + 1, name=name)
        if accept is None or accept(m):
            return m
    raise RuntimeError(f"no valid mesh for {name} seed {seed} after {MAX_ATTEMPTS} attempts")


def with_target_scale(m: Mesh, scale: float) -> Mesh:
    """Same mesh with the constant target W = scale * I (e.g. the equal-size
    target of eq. (3.1): scale = sqrt(|Omega| / N_E) in 2D)."""
    return replace(m, wkind=W_CONST, W=np.eye(m.dim) * float(scale))
