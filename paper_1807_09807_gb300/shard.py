"""Slab sharding of a structured order-k grid over ranks (one GPU each).

The objective and its derivatives are sums over elements (eq. (2.4) and the
Section 3.4 gradient and Hessian), so the elements can be split: rank r owns
the elements of a slab along the last axis (z in 3D, y in 2D) and evaluates
them with its own context over the slab's nodes. A node plane between two
slabs belongs to both local meshes:

* energy: each rank sums its own elements; F is the sum over ranks and
  min det A the minimum (one all-reduce each);
* gradient and Hessian action: each rank's local vector holds its elements'
  contributions, and one halo exchange per application adds the
  neighbour's contribution on each shared plane (send the plane, receive the
  neighbour's, add), after which every local vector equals the global one
  on the slab's nodes;
* dot products: each shared plane is counted by the lower rank only, then
  one all-reduce.

Only the host logic lives here (partition, local meshes, the exchange through
torch.distributed: NCCL between GPUs); the element kernels, the plane
additions and the dot products are the library's (tmop_vec_add,
tmop_vec_dot_segments), run on each rank's local mesh. The caller's vectors
are the local ones, [dim][local nodes]. The collectives take the plane
addition and the segment dot as arguments, so that the exchange logic can
also run on CPU ranks (gloo) with other arithmetic behind it.
"""
from __future__ import annotations

import math
from dataclasses import replace

import numpy as np

from . import meshgen as mg


class SlabPartition:
    """Elements split along the last axis into `world` contiguous slabs
    (sizes differing by at most one element)."""

    def __init__(self, dim: int, order: int, nx, world: int, rank: int):
        nx = tuple(int(v) for v in (nx if np.ndim(nx) else (nx,) * dim))
        if len(nx) != dim or world < 1 or not 0 <= rank < world or nx[-1] < world:
            raise ValueError("each rank needs at least one layer of elements")
        self.dim, self.order, self.nx, self.world, self.rank = dim, order, nx, world, rank
        base, extra = divmod(nx[-1], world)
        sizes = [base + (1 if r < extra else 0) for r in range(world)]
        self.e0 = sum(sizes[:rank])            # first element layer of this slab
        self.e1 = self.e0 + sizes[rank]        # one past the last
        self.N = [order * n + 1 for n in nx]   # global lattice points per axis
        self.plane = int(np.prod(self.N[:-1]))  # nodes per lattice plane of the last axis
        self.g0 = order * self.e0              # first and last lattice plane of the slab
        self.g1 = order * self.e1
        self.nplanes = self.g1 - self.g0 + 1
        self.nnode = self.plane * self.nplanes
        self.lo = rank > 0                     # plane g0 is shared with rank - 1
        self.hi = rank < world - 1             # plane g1 is shared with rank + 1

    @property
    def local_nx(self):
        return self.nx[:-1] + (self.e1 - self.e0,)

    def global_nodes(self) -> np.ndarray:
        """Global ids of the local nodes, in local order (the slab's planes)."""
        return np.arange(self.g0 * self.plane, (self.g1 + 1) * self.plane)

    def to_local(self, v_global: np.ndarray) -> np.ndarray:
        """[dim][global nnode] -> [dim][local nnode]"""
        return np.ascontiguousarray(v_global[:, self.g0 * self.plane:(self.g1 + 1) * self.plane])

    def local_mesh(self, m: mg.Mesh) -> mg.Mesh:
        """The slab as a mesh of its own: positions and fixed mask of the
        global mesh restricted to the slab's nodes (nodes of a shared plane
        keep the global mask: they stay free where the global mesh has them
        free), connectivity of the local structured grid."""
        _, en, _ = mg.structured(self.dim, self.order, self.local_nx)
        return replace(m, nx=self.local_nx, x=self.to_local(m.x), x_ideal=self.to_local(m.x_ideal),
                       elem_nodes=en, fixed=self.to_local(m.fixed))

    def owned(self) -> np.ndarray:
        """Per local node: 1 if this rank counts it in dot products (a shared
        plane is counted by the lower rank)."""
        w = np.ones(self.nnode, dtype=np.float64)
        if self.lo:
            w[:self.plane] = 0.0
        return w

    # -------------------------------------------------------------- collectives
    def halo_sum(self, y, dist, add=None):
        """Add the neighbours' contributions on the shared planes, in place.
        y: torch tensor [dim][local nnode] (on the device of the process
        group's backend). One exchange of whole planes with each neighbour;
        both sides add the same two partial sums, so the planes agree on both
        ranks. add(dst, src) adds a received plane of one component (default:
        tmop_vec_add on the GPU)."""
        import torch
        if add is None:
            from . import tmop as tm
            add = tm.vec_add
        P, d = self.plane, y.shape[0]
        reqs, recv = [], {}
        for side, peer, sl in (("lo", self.rank - 1, slice(0, P)), ("hi", self.rank + 1, slice(self.nnode - P, None))):
            if (side == "lo" and self.lo) or (side == "hi" and self.hi):
                send = y[:, sl].contiguous()
                buf = torch.empty_like(send)
                reqs.append(dist.isend(send, peer))
                reqs.append(dist.irecv(buf, peer))
                recv[side] = (sl, buf)
        for r in reqs:
            r.wait()
        for sl, buf in recv.values():
            for c in range(d):
                add(y[c, sl], buf[c])
        return y

    def dot(self, a, b, dist, seg_dot=None):
        """Global a . b of two halo-consistent local vectors [dim][local
        nnode]: the nodes this rank owns (all but a lower shared plane),
        summed over the ranks. seg_dot(a, b, first, count) returns the sum
        over the rows of a[:, first:first+count] . b[...] as a 1-element
        tensor (default: tmop_vec_dot_segments on the GPU)."""
        import torch
        first = self.plane if self.lo else 0
        count = self.nnode - first
        if seg_dot is None:
            from . import tmop as tm
            scratch = torch.empty(2048, dtype=torch.float64, device=a.device)
            out = torch.empty((), dtype=torch.float64, device=a.device)
            s = tm.vec_dot_segments(a, b, first, count, scratch, out).reshape(1)
        else:
            s = seg_dot(a, b, first, count).reshape(1)
        dist.all_reduce(s)
        return float(s.item())

    def energy(self, F_local: float, min_local: float, dist, device="cpu"):
        """(sum of the ranks' F, min of their min det A)."""
        import torch
        t = torch.tensor([F_local], dtype=torch.float64, device=device)
        m = torch.tensor([min_local], dtype=torch.float64, device=device)
        dist.all_reduce(t)
        dist.all_reduce(m, op=dist.ReduceOp.MIN)
        return float(t.item()), float(m.item())


class ShardedOperator:
    """The TMOP objective, gradient and Hessian action of a global structured
    mesh evaluated slab by slab: each rank runs the library's kernels on its
    local mesh and the collectives above make the results global."""

    def __init__(self, m: mg.Mesh, dist, precision=None, device="cuda"):
        from . import tmop as tm
        self.part = SlabPartition(m.dim, m.order, m.nx, dist.get_world_size(), dist.get_rank())
        self.mesh = self.part.local_mesh(m)
        self.ctx = tm.Context.from_mesh(self.mesh, precision=tm.FP64 if precision is None else precision)
        self.dist, self.device = dist, device

    def energy(self, x_local):
        rc, F, md = self.ctx.energy(x_local)
        return self.part.energy(F, md, self.dist, self.device)

    def gradient(self, x_local, out=None):
        g = self.ctx.gradient(x_local, out=out)
        return self.part.halo_sum(g, self.dist)

    def hess_apply(self, x_local, v_local, out=None):
        y = self.ctx.hess_apply(x_local, v_local, out=out)
        return self.part.halo_sum(y, self.dist)

    def dot(self, a, b):
        return self.part.dot(a, b, self.dist)

    def close(self):
        self.ctx.close()


# ------------------------------------------------------------------ Newton-MINRES on slabs
def _axpby_library(y, a, x, b):
    from . import tmop as tm
    tm.vec_axpby(y, a, x, b)


def sharded_minres(op, x, b, p, rtol=1e-10, maxit=2000, axpby=None):
    """MINRES (Paige and Saunders' recurrences, zero initial guess) for
    H(x) p = b on halo-consistent slab vectors: op.hess_apply gives H v with
    the shared planes summed, op.dot the global dot product, so every rank
    runs the same scalar recurrence on its slab. Stops when the residual
    estimate is at most rtol |b|. axpby(y, a, x, b): y = a x + b y (default:
    tmop_vec_axpby). Returns the iteration count."""
    import torch
    axpby = axpby or _axpby_library
    axpby(p, 0.0, b, 0.0)
    beta1 = math.sqrt(max(op.dot(b, b), 0.0))
    if beta1 == 0.0:
        return 0
    buf = [torch.empty_like(b) for _ in range(7)]
    r1, r2, t, v, w, w1, w2 = buf
    axpby(r1, 1.0, b, 0.0)
    axpby(r2, 1.0, b, 0.0)
    axpby(w, 0.0, b, 0.0)
    axpby(w1, 0.0, b, 0.0)
    axpby(w2, 0.0, b, 0.0)
    oldb, beta, dbar, epsln, phibar, cs, sn = 0.0, beta1, 0.0, 0.0, beta1, -1.0, 0.0
    itn = 0
    while itn < maxit:
        itn += 1
        axpby(v, 1.0 / beta, r2, 0.0)                  # Lanczos vector
        op.hess_apply(x, v, out=t)
        if itn >= 2:
            axpby(t, -beta / oldb, r1, 1.0)
        alfa = op.dot(v, t)
        axpby(t, -alfa / beta, r2, 1.0)
        r1, r2, t = r2, t, r1                          # rotate: r1 <- r2, r2 <- new
        oldb, beta = beta, math.sqrt(max(op.dot(r2, r2), 0.0))
        oldeps = epsln
        delta = cs * dbar + sn * alfa                  # previous rotation applied
        gbar = sn * dbar - cs * alfa
        epsln = sn * beta
        dbar = -cs * beta
        gamma = max(math.hypot(gbar, beta), 1e-300)    # next rotation
        cs, sn = gbar / gamma, beta / gamma
        phi, phibar = cs * phibar, sn * phibar
        w1, w2, w = w2, w, w1                          # new direction into the oldest buffer
        axpby(w, 1.0 / gamma, v, 0.0)
        axpby(w, -oldeps / gamma, w1, 1.0)
        axpby(w, -delta / gamma, w2, 1.0)
        axpby(p, phi, w, 1.0)
        if phibar <= rtol * beta1 or beta == 0.0:
            break
    return itn


def sharded_newton(op, x, max_newton=12, rtol=1e-12, krylov_rtol=1e-10, krylov_maxit=2000, f_factor=1.2,
                   g_factor=1.2, alpha_shrink=0.5, max_halvings=30, axpby=None):
    """Newton's method with the Section 3.4 line search over a slab-sharded
    mesh: the direction from sharded_minres (H p = g), trial x - alpha p,
    accepted when min det A > 0, F < f_factor F and |g| < g_factor |g|
    (alpha shrunk otherwise); stops when |g| <= rtol |g0|. op provides
    energy(x) -> (F, min det A), gradient(x, out), hess_apply(x, v, out)
    and dot(a, b), all global (ShardedOperator on GPUs). x (the local
    positions) is updated in place. Returns a report dict."""
    import torch
    axpby = axpby or _axpby_library
    rep = {"status": "ok", "iterations": 0, "krylov_iterations": 0, "alpha": 0.0}
    F, md = op.energy(x)
    if not md > 0.0:
        rep.update(status="inverted", F=F, min_detA=md)
        return rep
    xc, xt = x, torch.empty_like(x)
    g, gt, p = op.gradient(xc), torch.empty_like(x), torch.empty_like(x)
    gn = math.sqrt(max(op.dot(g, g), 0.0))
    gn0 = gn
    while True:
        if gn <= rtol * gn0:
            break
        if rep["iterations"] >= max_newton:
            rep["status"] = "iteration limit reached"
            break
        rep["krylov_iterations"] += sharded_minres(op, xc, g, p, krylov_rtol, krylov_maxit, axpby)
        alpha, accepted = 1.0, False
        for _ in range(max_halvings + 1):
            axpby(xt, 1.0, xc, 0.0)
            axpby(xt, -alpha, p, 1.0)
            Ft, mdt = op.energy(xt)
            if mdt > 0.0 and Ft < f_factor * F:
                op.gradient(xt, out=gt)
                gnt = math.sqrt(max(op.dot(gt, gt), 0.0))
                if gnt < g_factor * gn:
                    xc, xt, g, gt = xt, xc, gt, g
                    F, md, gn, accepted = Ft, mdt, gnt, True
                    break
            alpha *= alpha_shrink
        rep["iterations"] += 1
        if not accepted:
            rep["status"] = "line search exhausted"
            break
        rep["alpha"] = alpha
    if xc is not x:
        axpby(x, 1.0, xc, 0.0)
    rep.update(F=F, min_detA=md, grad_norm=gn, grad_norm0=gn0)
    return rep
