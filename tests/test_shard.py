"""Slab sharding (paper_1807_09807_gb300/shard.py) on CPU ranks over gloo:
every rank evaluates its own slab of elements (here with the FP64 oracle,
standing in for the rank's GPU kernels) and the partition's collectives --
the halo sum of the shared node planes, the all-reduced energy and minimum,
the owned-node dot product -- must reproduce the single-rank results."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

from paper_1807_09807_gb300 import meshgen as mg   # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


CASES = {"3d": ("c4", dict(nx=(3, 2, 5))), "2d": ("c2", dict(nx=(4, 7)))}


def _rank(rank, ws, port, case, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import oracle
    from paper_1807_09807_gb300.shard import SlabPartition
    name, kw = CASES[case]
    m = mg.make_mesh(name, 3, **kw)
    part = SlabPartition(m.dim, m.order, m.nx, ws, rank)
    lm = part.local_mesh(m)
    orc = oracle.Problem(lm.dim, lm.order, lm.elem_nodes, lm.nnode, lm.fixed, lm.nq, lm.metric)
    v = np.random.default_rng(11).standard_normal(m.x.shape) * (1 - m.fixed)
    _, F, md = orc.energy(lm.x)
    F, md = part.energy(F, md, dist)
    add = lambda dst, src: dst.add_(src)          # noqa: E731  (CPU stand-ins for the library's kernels)
    seg = lambda a, b, i, n: (a[:, i:i + n] * b[:, i:i + n]).sum()  # noqa: E731
    g = part.halo_sum(torch.tensor(orc.gradient(lm.x)), dist, add)
    hv = part.halo_sum(torch.tensor(orc.hess_apply(lm.x, part.to_local(v))), dist, add)
    gg = part.dot(g, g, dist, seg)
    vhv = part.dot(torch.tensor(part.to_local(v)), hv, dist, seg)
    out.put((rank, F, md, g.numpy(), hv.numpy(), gg, vhv))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case,ws", [("3d", 2), ("3d", 3), ("2d", 2)])
def test_slab_sharding_reproduces_the_single_rank_operator(case, ws):
    import oracle
    from paper_1807_09807_gb300.shard import SlabPartition
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, case, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(ws)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    name, kw = CASES[case]
    m = mg.make_mesh(name, 3, **kw)
    orc = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, m.metric)
    v = np.random.default_rng(11).standard_normal(m.x.shape) * (1 - m.fixed)
    _, F, md = orc.energy(m.x)
    g, hv = orc.gradient(m.x), orc.hess_apply(m.x, v)
    covered = np.zeros(m.nnode, dtype=int)
    for rank, Fr, mdr, gr, hvr, ggr, vhvr in res:
        part = SlabPartition(m.dim, m.order, m.nx, ws, rank)
        assert abs(Fr - F) <= 1e-13 * F and mdr == md
        np.testing.assert_allclose(gr, part.to_local(g), rtol=0, atol=1e-13 * np.abs(g).max())
        np.testing.assert_allclose(hvr, part.to_local(hv), rtol=0, atol=1e-13 * np.abs(hv).max())
        assert abs(ggr - float((g * g).sum())) <= 1e-12 * float((g * g).sum())
        assert abs(vhvr - float((v * hv).sum())) <= 1e-12 * abs(float((v * hv).sum()))
        covered[part.global_nodes()] += part.owned().astype(int)
    assert np.all(covered == 1)          # every node counted once in the dot products


def _axpby_cpu(y, a, x, b):
    # the CPU stand-in of tmop_vec_axpby (b = 0: y's old contents unread)
    y.copy_(a * x if b == 0.0 else a * x + b * y)


class _OracleSlabOp:
    """One rank's slab evaluated by the FP64 oracle (standing in for the
    rank's GPU kernels), made global by the partition's collectives: the
    operator interface sharded_newton drives."""

    def __init__(self, part, lm):
        import oracle
        self.part = part
        self.orc = oracle.Problem(lm.dim, lm.order, lm.elem_nodes, lm.nnode, lm.fixed, lm.nq, lm.metric)
        self.add = lambda dst, src: dst.add_(src)                          # noqa: E731
        self.seg = lambda a, b, i, n: (a[:, i:i + n] * b[:, i:i + n]).sum()  # noqa: E731

    def energy(self, x):
        _, F, md = self.orc.energy(x.numpy())
        return self.part.energy(F, md, dist)

    def _put(self, val, out):
        t = self.part.halo_sum(torch.tensor(val), dist, self.add)
        if out is None:
            return t
        out.copy_(t)
        return out

    def gradient(self, x, out=None):
        return self._put(self.orc.gradient(x.numpy()), out)

    def hess_apply(self, x, v, out=None):
        return self._put(self.orc.hess_apply(x.numpy(), v.numpy()), out)

    def dot(self, a, b):
        return self.part.dot(a, b, dist, self.seg)


class _DenseOp:
    """A dense symmetric matrix acting on [2][n/2] vectors, for the MINRES
    recurrences alone (no partition, no collectives)."""

    def __init__(self, A):
        self.A = torch.tensor(A)

    def hess_apply(self, x, v, out=None):
        out.copy_((self.A @ v.reshape(-1)).reshape(v.shape))
        return out

    def dot(self, a, b):
        return float((a * b).sum())


def test_sharded_minres_solves_symmetric_indefinite_systems():
    """sharded_minres against a dense solve: a symmetric indefinite matrix
    (MINRES's case, where CG would not apply), a positive definite one, and a
    zero right-hand side (p = 0, no iteration)."""
    from paper_1807_09807_gb300.shard import sharded_minres
    rng = np.random.default_rng(5)
    Qm, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    for eig in (np.concatenate([-np.linspace(1, 3, 15), np.linspace(0.5, 4, 25)]), np.linspace(0.2, 5, 40)):
        A = (Qm * eig) @ Qm.T
        b = torch.tensor(rng.standard_normal((2, 20)))
        p = torch.empty_like(b)
        it = sharded_minres(_DenseOp(A), None, b, p, rtol=1e-13, maxit=200, axpby=_axpby_cpu)
        ref = np.linalg.solve(A, b.numpy().reshape(-1))
        assert 0 < it <= 200
        assert np.linalg.norm(p.numpy().reshape(-1) - ref) <= 1e-10 * np.linalg.norm(ref)
    p = torch.full((2, 20), 7.0)
    assert sharded_minres(_DenseOp(A), None, torch.zeros(2, 20), p, axpby=_axpby_cpu) == 0
    assert torch.equal(p, torch.zeros(2, 20))


NEWTON_CASE = ("c3", dict(nx=(2, 2, 6)))


def _newton_rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from paper_1807_09807_gb300.shard import SlabPartition, sharded_newton
    name, kw = NEWTON_CASE
    m = mg.make_mesh(name, 4, **kw)
    part = SlabPartition(m.dim, m.order, m.nx, ws, rank)
    lm = part.local_mesh(m)
    x = torch.tensor(lm.x)
    rep = sharded_newton(_OracleSlabOp(part, lm), x, axpby=_axpby_cpu)
    out.put((rank, rep, x.numpy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_sharded_newton_reaches_the_single_rank_minimiser(ws):
    """Newton-MINRES with the det A > 0 line search on slab vectors (the
    global dots and the halo sums of each product), 2 and 3 gloo ranks:
    converged, with the F and the nodes of the oracle's single-rank Newton."""
    import oracle
    from paper_1807_09807_gb300.shard import SlabPartition
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_newton_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=600) for _ in range(ws)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    name, kw = NEWTON_CASE
    m = mg.make_mesh(name, 4, **kw)
    orc = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, m.metric)
    rc, xo, hist = orc.newton(m.x, max_newton=12)
    assert rc == oracle.OK
    F0 = hist[0, 0]
    for rank, rep, xr in res:
        assert rep["status"] == "ok" and rep["grad_norm"] <= 1e-12 * rep["grad_norm0"], rep
        assert abs(rep["F"] - hist[-1, 0]) <= 1e-12 * F0 and rep["min_detA"] > 0
        assert rep["F"] == res[0][1]["F"] and rep["iterations"] == res[0][1]["iterations"]
        xl = SlabPartition(m.dim, m.order, m.nx, ws, rank).to_local(xo)
        assert np.abs(xr - xl).max() <= 1e-9 * np.abs(xo).max()


def test_slab_partition_shapes():
    from paper_1807_09807_gb300.shard import SlabPartition
    parts = [SlabPartition(3, 3, (4, 4, 10), 4, r) for r in range(4)]
    assert [p.e1 - p.e0 for p in parts] == [3, 3, 2, 2]
    assert parts[0].g0 == 0 and parts[-1].g1 == 30 and all(a.g1 == b.g0 for a, b in zip(parts, parts[1:]))
    assert [p.lo for p in parts] == [False, True, True, True] and [p.hi for p in parts] == [True, True, True, False]
    with pytest.raises(ValueError):
        SlabPartition(3, 3, (4, 4, 2), 3, 0)


@pytest.mark.gpu
def test_sharded_operator_single_rank_gpu_and_vector_helpers():
    """On one GPU (a one-rank NCCL group) the sharded operator is the
    context's own operator, and the library's plane add and segment dot
    (tmop_vec_add, tmop_vec_dot_segments) match their definitions."""
    from paper_1807_09807_gb300 import build as cuda_build
    cuda_build.build()
    from paper_1807_09807_gb300 import tmop as tm
    from paper_1807_09807_gb300.shard import ShardedOperator
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()), RANK="0", WORLD_SIZE="1")
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        m = mg.make_mesh("c4", 2, nx=(3, 3, 4))
        op = ShardedOperator(m, dist)
        ctx = tm.Context.from_mesh(m)
        x = torch.tensor(m.x, device="cuda")
        v = torch.tensor(np.random.default_rng(2).standard_normal(m.x.shape), device="cuda")
        assert op.energy(x) == ctx.energy(x)[1:]
        g1, g2 = op.gradient(x).cpu().numpy(), ctx.gradient(x).cpu().numpy()
        assert np.abs(g1 - g2).max() <= 1e-13 * np.abs(g2).max()
        y1, y2 = op.hess_apply(x, v).cpu().numpy(), ctx.hess_apply(x, v).cpu().numpy()
        assert np.abs(y1 - y2).max() <= 1e-13 * np.abs(y2).max()
        a = torch.tensor(np.random.default_rng(3).standard_normal((3, 1000)), device="cuda")
        b = torch.tensor(np.random.default_rng(4).standard_normal((3, 1000)), device="cuda")
        out = torch.empty((), dtype=torch.float64, device="cuda")
        tm.vec_dot_segments(a, b, 17, 900, torch.empty(2048, dtype=torch.float64, device="cuda"), out)
        ref = float((a[:, 17:917] * b[:, 17:917]).sum().item())
        assert abs(out.item() - ref) <= 1e-13 * abs(ref) + 1e-12
        y = a.clone()
        tm.vec_add(y[1], b[1].contiguous())
        assert torch.equal(y[1], a[1] + b[1]) and torch.equal(y[0], a[0])
        z = torch.full_like(a, float("nan"))
        tm.vec_axpby(z, 2.5, a, 0.0)                       # b = 0: z's old contents unread
        assert torch.equal(z, 2.5 * a)
        tm.vec_axpby(z, -0.5, b, 3.0)
        assert torch.allclose(z, 7.5 * a - 0.5 * b, rtol=1e-15, atol=1e-15)
        # Newton-MINRES on the sharded operator (one rank): the context's own Newton's F
        from paper_1807_09807_gb300.shard import sharded_newton
        xs = x.clone()
        rep = sharded_newton(op, xs)
        r = ctx.newton_solve(x.clone(), max_newton=12)
        assert rep["status"] == "ok" and r.status == tm.OK
        assert abs(rep["F"] - r.report["F"]) <= 1e-12 * ctx.energy(x)[1] and rep["min_detA"] > 0
        op.close()
    finally:
        dist.destroy_process_group()
