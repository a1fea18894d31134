"""GPU parity: every C-ABI call of the CUDA library against the FP64 CPU
oracle on the same seeded inputs.

Tolerances (FP64 path, relative):
  F and min det A: 1e-12; gradient and Hessian action: normwise 1e-12
  (FP64 atomics make the summation order of nodal contributions differ from
  the oracle's element order, so entries agree only normwise).
FP32-mixed path: bounds derived from eps32 = 6e-8 times the conditioning of
each result; see test_fp32_mixed_bounds.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1807_09807_gb300 import meshgen as mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def tm():
    from paper_1807_09807_gb300 import build as cuda_build
    cuda_build.build()
    from paper_1807_09807_gb300 import tmop
    tmop.load()
    return tmop


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def orc_for(m, metric=None, W=None, Wqp=None):
    if Wqp is not None:
        return oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, metric or m.metric,
                              quad_kind=m.quad_kind, wkind=oracle.W_PER_QP, W=Wqp)
    wk = oracle.W_IDENTITY if W is None else oracle.W_CONST
    return oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, metric or m.metric,
                          quad_kind=m.quad_kind, wkind=wk, W=W)


def make(name, seed=1, **kw):
    """Seeded mesh, redrawn until the oracle sees det A > 0 everywhere."""
    return mg.make_mesh(name, seed, accept=lambda mm: orc_for(mm).energy(mm.x)[2] > 0, **kw)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def check_all(tm, m, ctx, orc, rtol_F=RTOL, rtol_vec=RTOL, seed=0):
    x = dev(m.x)
    rc, F, md = ctx.energy(x)
    rco, Fo, mdo = orc.energy(m.x)
    assert rc == tm.OK and rco == oracle.OK
    assert abs(F - Fo) <= rtol_F * abs(Fo), (F, Fo)
    assert abs(md - mdo) <= rtol_F * abs(mdo), (md, mdo)
    g = host(ctx.gradient(x))
    go = orc.gradient(m.x)
    assert rel(g, go) <= rtol_vec, rel(g, go)
    assert np.all(g[m.fixed == 1] == 0.0)
    # the one-pass energy + gradient of the line search: the same F, min det A
    # and g up to the order of the sums
    g2, F2, md2 = ctx.energy_gradient(x)
    assert abs(F2.item() - F) <= 1e-13 * abs(F) and md2.item() == md
    assert rel(host(g2), g) <= 1e-13
    v = np.random.default_rng(seed).standard_normal(m.x.shape)
    y = host(ctx.hess_apply(x, dev(v)))
    yo = orc.hess_apply(m.x, v)
    assert rel(y, yo) <= rtol_vec, rel(y, yo)
    assert np.all(y[m.fixed == 1] == 0.0)
    # the gradient and the Hessian action in one call (one element pass where
    # the context allows): the two kernels' results up to the order of the
    # sums, and the oracle's
    gf, yf = (host(t) for t in ctx.gradient_hess_apply(x, dev(v)))
    assert rel(gf, g) <= 1e-13 and rel(yf, y) <= 1e-13, (rel(gf, g), rel(yf, y))
    assert rel(gf, go) <= rtol_vec and rel(yf, yo) <= rtol_vec
    assert np.all(gf[m.fixed == 1] == 0.0) and np.all(yf[m.fixed == 1] == 0.0)
    return F, g, y


SMALL = [("c1", {}), ("c2", dict(nx=6)), ("c3", dict(nx=3)), ("c4", dict(nx=3)), ("c5", dict(nx=5))]


@pytest.mark.parametrize("name,kw", SMALL)
@pytest.mark.parametrize("structured", [True, False])
def test_fp64_small_configs(tm, name, kw, structured):
    m = make(name, 1, **kw)
    check_all(tm, m, tm.Context.from_mesh(m, structured=structured), orc_for(m))


@pytest.mark.parametrize("dim,metric", [(2, 1), (2, 2), (2, 7), (2, 9), (2, 14), (2, 77), (2, 98),
                                        (3, 1), (3, 14), (3, 98), (3, 302), (3, 303)])
def test_fp64_every_metric(tm, dim, metric):
    m = make("c1" if dim == 2 else "c3", 2, nx=4 if dim == 2 else 2)
    scale = 1.0 / 4 if metric in (7, 9, 77) else None      # element size: W2 of eq. (3.1)
    ctx = tm.Context.from_mesh(m, metric=metric, target_scale=scale)
    orc = orc_for(m, metric=metric, W=None if scale is None else np.eye(dim) * scale)
    check_all(tm, m, ctx, orc)


@pytest.mark.parametrize("dim,order,nq", [(2, 1, 2), (2, 1, 3), (2, 2, 3), (2, 2, 5), (2, 3, 4), (2, 3, 6),
                                          (2, 4, 5), (2, 4, 6), (3, 1, 2), (3, 1, 3), (3, 2, 3), (3, 3, 4),
                                          (3, 4, 5), (3, 4, 6)])
def test_fp64_every_order_and_rule(tm, dim, order, nq):
    m = make("c1" if dim == 2 else "c3", 3, order=order, nq=nq, nx=3 if dim == 2 else 2)
    check_all(tm, m, tm.Context.from_mesh(m), orc_for(m))


def test_fp64_gauss_lobatto(tm):
    m = make("c2", 1, nx=5, quad_kind=mg.GLL, nq=6)
    check_all(tm, m, tm.Context.from_mesh(m), orc_for(m))


@pytest.mark.parametrize("dim", [2, 3])
def test_fp64_general_and_per_point_targets(tm, dim):
    rng = np.random.default_rng(7)
    m = make("c1" if dim == 2 else "c3", 4, nx=3 if dim == 2 else 2)
    W = (np.eye(dim) + 0.2 * rng.standard_normal((dim, dim))) / 6
    if np.linalg.det(W) < 0:
        W[:, 0] *= -1
    m.W = W
    check_all(tm, m, tm.Context.from_mesh(m), orc_for(m, W=W))
    Wq = (np.eye(dim) + 0.15 * rng.standard_normal((m.nelem, m.Q, dim, dim))) / 6
    Wq[np.linalg.det(Wq) < 0, :, 0] *= -1
    m.W = None
    check_all(tm, m, tm.Context.from_mesh(m, W_per_qp=Wq), orc_for(m, Wqp=Wq))


@pytest.mark.parametrize("dim,structured", [(2, True), (2, False), (3, True), (3, False)])
def test_jacobians_match_oracle(tm, dim, structured):
    """A(x) at every quadrature point (eq. (2.2)) against the oracle's."""
    m = make("c1" if dim == 2 else "c3", 5, nx=(3, 2) if dim == 2 else (2, 3, 1))
    J = host(tm.Context.from_mesh(m, structured=structured).jacobians(dev(m.x)))
    Jo = orc_for(m).jacobians(m.x)
    assert np.abs(J - Jo).max() <= 1e-13 * np.abs(Jo).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_targets_from_positions_match_oracle(tm, dim):
    """W2 (eq. (3.1)), W3 (Section 3.1) and W0 (Section 4.3.2) built on the
    GPU from x0, against the oracle run with the same targets written out
    from its own Jacobians of x0."""
    m = make("c1" if dim == 2 else "c3", 6, nx=3 if dim == 2 else 2)
    Jo = orc_for(m).jacobians(m.x)
    w, _ = orc_for(m).tables()
    dets = np.linalg.det(Jo)
    alpha = float(np.sum(dets * w[None, :])) / m.nelem
    cases = [
        (tm.WT_EQUAL_SIZE, dict(W=alpha ** (1.0 / dim) * np.eye(dim))),
        (tm.WT_LOCAL_SIZE, dict(Wqp=(dets ** (1.0 / dim))[:, :, None, None] * np.eye(dim))),
        (tm.WT_INITIAL, dict(Wqp=Jo)),
    ]
    x1 = m.x + 0.02 / (m.order * 3) * np.random.default_rng(1).uniform(-1, 1, m.x.shape) * (1 - m.fixed)
    for kind, wk in cases:
        for metric in ((2, 98) if dim == 2 else (303, 98)):
            ctx = tm.Context.from_mesh(m, metric=metric)
            ctx.set_targets_from_positions(kind, dev(m.x))
            orc = orc_for(m, metric=metric, **wk)
            check_all(tm, dataclasses.replace(m, x=x1), ctx, orc)


def test_replication_metric_on_gpu(tm):
    """Section 4.3.2 on the GPU: mu98 with W0 = A(x_init) gives F = 0, g = 0
    at x_init, and Newton from a perturbed mesh returns to x_init; the gamma
    blend mu98(A W0^-1) + (gamma / (1 - gamma)) mu2(A) converges to the
    oracle's minimiser."""
    m = make("c1", 1, nx=4)
    ctx = tm.Context.from_mesh(m, metric=98)
    x0 = dev(m.x)
    ctx.set_targets_from_positions(tm.WT_INITIAL, x0)
    rc, F, md = ctx.energy(x0)
    assert rc == tm.OK and abs(F) < 1e-13
    assert np.abs(host(ctx.gradient(x0))).max() < 1e-12
    x1 = m.x + 0.05 / (m.order * 4) * np.random.default_rng(2).uniform(-1, 1, m.x.shape) * (1 - m.fixed)
    x = dev(x1)
    res = ctx.newton_solve(x, max_newton=20)
    assert res.status == tm.OK and np.abs(host(x) - m.x).max() < 1e-10
    gamma = 0.3
    eta = np.full((m.nelem, m.Q), gamma / (1 - gamma))
    ctx.set_composite(2, np.eye(2), eta)
    x = dev(m.x)
    res = ctx.newton_solve(x, max_newton=30)
    orc = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, 98, wkind=oracle.W_PER_QP,
                         W=orc_for(m).jacobians(m.x), metric2=2, eta2=eta)
    rco, xo, _ = orc.newton(m.x, max_newton=30)
    assert res.status == tm.OK and rco == oracle.OK
    assert np.abs(host(x) - xo).max() < 1e-10 * np.abs(xo).max()
    assert np.linalg.norm(xo - m.x) > 1e-3


def test_targets_from_inverted_positions_are_rejected(tm):
    m = make("c1", 1, nx=3)
    ctx = tm.Context.from_mesh(m, metric=98)
    xb = m.x.copy()
    xb[0] = -xb[0]                         # mirrored mesh: det A < 0 everywhere
    for kind in (tm.WT_LOCAL_SIZE, tm.WT_INITIAL, tm.WT_EQUAL_SIZE):
        with pytest.raises(tm.TmopError) as ei:
            ctx.set_targets_from_positions(kind, dev(xb))
        assert ei.value.status == tm.ERR_INVERTED
    # targets unchanged: still W = I
    check_all(tm, m, ctx, orc_for(m, metric=98))


def test_fp64_ragged_and_single_element(tm):
    # one element, and a 5x3 (non-square, element count not a multiple of a block)
    for nx in [1, (5, 3)]:
        m = make("c1", 1, nx=nx)
        check_all(tm, m, tm.Context.from_mesh(m), orc_for(m))
    m = make("c3", 1, nx=(3, 2, 1))
    check_all(tm, m, tm.Context.from_mesh(m), orc_for(m))


def test_fp64_tangential_relaxation(tm):
    """Per-component fixed mask: boundary nodes slide along axis-parallel faces
    (Section 4.1); parity, and Newton keeps them on their faces."""
    for name, kw in [("c1", dict(nx=4)), ("c3", dict(nx=3))]:
        m = make(name, 3, tangential=True, **kw)
        ctx = tm.Context.from_mesh(m)
        check_all(tm, m, ctx, orc_for(m))
        x = dev(m.x)
        r = ctx.newton_solve(x, max_newton=20)
        assert r.status == tm.OK
        xf = host(x)
        assert np.array_equal(xf[m.fixed == 1], m.x[m.fixed == 1])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_all_dofs_fixed_and_zero_rhs(tm, prec):
    """Degenerate cases: a mesh whose nodes are all on the boundary (one
    order-1 element, 2D and 3D) has no free dof, so the gradient and every
    Hessian action vanish and Newton stops at once with x unchanged; a
    Krylov solve with b = 0 returns p = 0."""
    for name, nx in (("c1", 1), ("c3", (1, 1, 1))):
        m = make(name, 1, order=1, nq=2, nx=nx)
        assert np.all(m.fixed == 1)
        ctx = tm.Context.from_mesh(m, precision=tm.FP64 if prec == "fp64" else tm.FP32_MIXED)
        x = dev(m.x)
        assert np.all(host(ctx.gradient(x)) == 0.0)
        v = dev(np.random.default_rng(0).standard_normal(m.x.shape))
        assert np.all(host(ctx.hess_apply(x, v)) == 0.0)
        gf, yf = ctx.gradient_hess_apply(x, v)
        assert np.all(host(gf) == 0.0) and np.all(host(yf) == 0.0)
        ctx.linearize(x)
        assert np.all(host(ctx.hess_apply_pa(v)) == 0.0)
        res = ctx.newton_solve(x, max_newton=5)
        assert res.status == tm.OK and res.report["iterations"] == 0
        assert np.array_equal(host(x), m.x)
    m = make("c1", 1, nx=3)
    ctx = tm.Context.from_mesh(m)
    p, it = ctx.krylov_solve(dev(m.x), dev(np.zeros_like(m.x)))
    assert np.all(host(p) == 0.0) and it >= 0


def test_fp64_no_fixed_dofs(tm):
    m = make("c1", 1, nx=3)
    m.fixed = np.zeros_like(m.fixed)
    check_all(tm, m, tm.Context.from_mesh(m), orc_for(m))


@pytest.mark.parametrize("name,metric", [("c2", 2), ("c2", 7), ("c3", 303), ("c3", 302)])
def test_fp64_full_size(tm, name, metric):
    m = make(name, 1)
    scale = 1.0 / 64 if metric == 7 else None              # element size: W2 of eq. (3.1)
    check_all(tm, m, tm.Context.from_mesh(m, metric=metric, target_scale=scale),
              orc_for(m, metric=metric, W=None if scale is None else np.eye(2) * scale))


def _patch(m, nodes):
    """Elements touching any of the given nodes."""
    return np.nonzero(np.isin(m.elem_nodes, nodes).any(axis=1))[0].astype(np.int32)


def test_fp64_full_c4_sampled(tm):
    """48^3 order-3 hexes (the benchmark workload, same launch shapes): F and
    min det A in full; gradient and Hessian action at 64 sampled free nodes,
    each against the oracle restricted to the elements around them."""
    m = make("c4", 1)
    ctx = tm.Context.from_mesh(m)
    orc = orc_for(m)
    x = dev(m.x)
    rc, F, md = ctx.energy(x)
    _, Fo, mdo = orc.energy(m.x)
    assert abs(F - Fo) <= RTOL * Fo and abs(md - mdo) <= RTOL * abs(mdo)
    rng = np.random.default_rng(3)
    free = np.nonzero(m.fixed[0] == 0)[0]
    nodes = rng.choice(free, 64, replace=False)
    els = _patch(m, nodes)
    g = host(ctx.gradient(x))[:, nodes]
    go = orc.gradient(m.x, elems=els)[:, nodes]
    assert rel(g, go) <= RTOL
    v = rng.standard_normal(m.x.shape)
    y = host(ctx.hess_apply(x, dev(v)))[:, nodes]
    yo = orc.hess_apply(m.x, v, elems=els)[:, nodes]
    assert rel(y, yo) <= RTOL
    # the fused gradient + Hessian action in the launch shape bench.py times
    gf, yf = ctx.gradient_hess_apply(x, dev(v))
    assert rel(host(gf)[:, nodes], go) <= RTOL and rel(host(yf)[:, nodes], yo) <= RTOL
    emin = host(ctx.element_min_detA(x))
    sub = rng.choice(m.nelem, 200, replace=False).astype(np.int32)
    for e in sub[:20]:
        _, _, mde = orc.energy(m.x, elems=np.array([e], dtype=np.int32))
        assert abs(emin[e] - mde) <= RTOL * abs(mde)
    assert abs(emin.min() - mdo) <= RTOL * abs(mdo)


def test_fp32_compact_product_full_c4_sampled(tm):
    """The benchmark's FP32 Krylov operator at full size (48^3 order-3 hexes,
    compact records, the launch shape bench.py times): the stored-Hessian
    product at 64 sampled free nodes against the oracle restricted to the
    elements around them, within the FP32 bound of the other FP32 products;
    and the same product from the FP64 context's packed Hessians at 1e-12."""
    m = make("c4", 1)
    orc = orc_for(m)
    x = dev(m.x)
    rng = np.random.default_rng(4)
    free = np.nonzero(m.fixed[0] == 0)[0]
    nodes = rng.choice(free, 64, replace=False)
    els = _patch(m, nodes)
    v = rng.standard_normal(m.x.shape)
    yo = orc.hess_apply(m.x, v, elems=els)[:, nodes]
    c32 = tm.Context.from_mesh(m, precision=tm.FP32_MIXED)
    c32.linearize(x)
    assert c32.pa_layout()[0] == 14
    assert rel(host(c32.hess_apply_pa(dev(v)))[:, nodes], yo) <= 1e-5
    c32.close()
    c64 = tm.Context.from_mesh(m)
    c64.linearize(x)
    assert rel(host(c64.hess_apply_pa(dev(v)))[:, nodes], yo) <= RTOL


def test_fp32_hessian_step_full_c4_sampled(tm):
    """The FP32-Hessian form of the benchmark step at full size (48^3
    order-3 hexes, the launch shapes bench.py times): the FP64 gradient and
    the fused FP64 energy + gradient of the line search at 1e-12, and the
    FP32 Hessian action recomputed from x (matrix-free) within the FP32
    bound, at 64 sampled free nodes against the oracle restricted to the
    elements around them."""
    m = make("c4", 1)
    orc = orc_for(m)
    x = dev(m.x)
    rng = np.random.default_rng(6)
    free = np.nonzero(m.fixed[0] == 0)[0]
    nodes = rng.choice(free, 64, replace=False)
    els = _patch(m, nodes)
    v = rng.standard_normal(m.x.shape)
    go = orc.gradient(m.x, elems=els)[:, nodes]
    yo = orc.hess_apply(m.x, v, elems=els)[:, nodes]
    _, Fo, mdo = orc.energy(m.x)
    c = tm.Context.from_mesh(m, precision=tm.FP32_MIXED)
    assert rel(host(c.gradient(x))[:, nodes], go) <= RTOL
    g, F, md = c.energy_gradient(x)
    assert rel(host(g)[:, nodes], go) <= RTOL
    assert abs(float(F) - Fo) <= RTOL * Fo and abs(float(md) - mdo) <= RTOL * abs(mdo)
    assert rel(host(c.hess_apply(x, dev(v)))[:, nodes], yo) <= 1e-5
    c.close()


def test_fp32_packed_product_full_c4_sampled(tm):
    """The 45-value FP32 product at full size, as bench.py times it: mu302
    (not written in |T|^2 and det T, so the packed A-space Hessians are
    stored) on the 48^3 order-3 mesh, at 64 sampled free nodes against the
    oracle restricted to the elements around them, within the FP32 bound."""
    m = make("c4", 1)
    orc = orc_for(m, metric=302)
    x = dev(m.x)
    rng = np.random.default_rng(5)
    free = np.nonzero(m.fixed[0] == 0)[0]
    nodes = rng.choice(free, 64, replace=False)
    els = _patch(m, nodes)
    v = rng.standard_normal(m.x.shape)
    yo = orc.hess_apply(m.x, v, elems=els)[:, nodes]
    c32 = tm.Context.from_mesh(m, precision=tm.FP32_MIXED, metric=302)
    c32.linearize(x)
    assert c32.pa_layout()[0] == 45
    assert rel(host(c32.hess_apply_pa(dev(v)))[:, nodes], yo) <= 1e-5


def test_inverted_mesh(tm):
    m = make("c1", 1, nx=4)
    x = m.x_ideal.copy()
    node = m.elem_nodes[5, 4]
    x[0, node] += 0.3
    ctx = tm.Context.from_mesh(m)
    rc, F, md = ctx.energy(dev(x))
    rco, Fo, mdo = orc_for(m).energy(x)
    assert rc == tm.ERR_INVERTED and rco == oracle.ERR_INVERTED
    assert F == np.inf and abs(md - mdo) <= RTOL * abs(mdo)
    em = host(ctx.element_min_detA(dev(x)))
    assert (em <= 0).sum() >= 1 and np.all((em <= 0) == (np.array(
        [orc_for(m).energy(x, elems=np.array([e], dtype=np.int32))[2] for e in range(m.nelem)]) <= 0))


def test_deterministic_energy(tm):
    m = make("c3", 1, nx=8)
    ctx = tm.Context.from_mesh(m)
    x = dev(m.x)
    vals = {ctx.energy(x)[1] for _ in range(5)}
    assert len(vals) == 1


def test_fused_gradient_hessian_action_fallbacks_and_arguments(tm):
    """Contexts the one-pass kernel does not cover (restricted movement,
    deterministic sums, the FP32-mixed form) run the two kernels and give
    their results; g and y must be distinct."""
    m = make("c3", 6, nx=2)
    x = dev(m.x)
    v = dev(np.random.default_rng(6).standard_normal(m.x.shape))
    orc = orc_for(m)
    for setup in ("delta", "det", "fp32"):
        ctx = tm.Context.from_mesh(m, precision=tm.FP32_MIXED if setup == "fp32" else tm.FP64)
        if setup == "delta":
            ctx.set_restricted_movement(20.0, dev(m.x * 0.99))
        if setup == "det":
            ctx.set_deterministic(True)
        g, y = ctx.gradient(x), ctx.hess_apply(x, v)
        gf, yf = ctx.gradient_hess_apply(x, v)
        if setup == "det":
            assert torch.equal(gf, g) and torch.equal(yf, y)
        assert rel(host(gf), host(g)) <= 1e-13 and rel(host(yf), host(y)) <= 1e-13
        if setup == "fp32":
            assert rel(host(gf), orc.gradient(m.x)) <= RTOL
            assert rel(host(yf), orc.hess_apply(m.x, host(v))) <= 1e-5
    ctx = tm.Context.from_mesh(m)
    same = torch.empty_like(x)
    with pytest.raises(tm.TmopError):
        ctx.gradient_hess_apply(x, v, g=same, y=same)


# ---------------------------------------------------------------- composite metrics
@pytest.mark.parametrize("dim,ma,mb,prec", [(2, 1, 77, "fp64"), (2, 2, 7, "fp64"), (3, 303, 14, "fp64"),
                                            (3, 303, 302, "fp64"), (3, 303, 14, "fp32")])
def test_composite_metric_matches_oracle(tm, dim, ma, mb, prec):
    """eq. (4.1): mu_a(A W^-1) + eta_q mu_b(A W2^-1) with per-point weights and
    a non-symmetric W2: energy, gradient, recompute and partially assembled
    Hessian actions against the oracle."""
    rng = np.random.default_rng(dim * 100 + mb)
    m = make("c1" if dim == 2 else "c3", 4, nx=4 if dim == 2 else 3)
    W2 = (np.eye(dim) + 0.15 * rng.standard_normal((dim, dim))) * 0.3
    if np.linalg.det(W2) < 0:
        W2[:, 0] *= -1
    eta = 0.5 + rng.random((m.nelem, m.Q))
    ctx = tm.Context.from_mesh(m, metric=ma, precision=tm.FP64 if prec == "fp64" else tm.FP32_BULK)
    ctx.set_composite(mb, W2, eta)
    orc = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, ma, metric2=mb, W2=W2, eta2=eta)
    tol_F, tol_v = (RTOL, RTOL) if prec == "fp64" else (1e-6, 1e-5)
    check_all(tm, m, ctx, orc, rtol_F=tol_F, rtol_vec=tol_v)
    x = dev(m.x)
    ctx.linearize(x)
    v = rng.standard_normal(m.x.shape)
    assert rel(host(ctx.hess_apply_pa(dev(v))), orc.hess_apply(m.x, v)) <= tol_v
    ctx.set_composite(0)
    assert abs(ctx.energy(x)[1] - _single(m, ma).energy(m.x)[1]) <= tol_F * _single(m, ma).energy(m.x)[1]


def _single(m, metric):
    return oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, metric)


# ---------------------------------------------------------------- restricted movement
@pytest.mark.parametrize("name,kw,metric,prec", [("c1", dict(nx=4), 2, "fp64"), ("c2", dict(nx=5), 2, "fp64"),
                                                 ("c3", dict(nx=3), 303, "fp64"), ("c4", dict(nx=2), 303, "fp64"),
                                                 ("c3", dict(nx=3), 303, "mixed")])
def test_restricted_movement_matches_oracle(tm, name, kw, metric, prec):
    """eq. (4.2): + sum_E int delta |x - x_init|^2: energy, gradient, recompute
    and partially assembled Hessian actions against the oracle, and a Newton
    solve that stays closer to x_init than without the term."""
    m = make(name, 2, **kw)
    rng = np.random.default_rng(7)
    x_init = m.x + 0.02 / (m.order * m.nx[0]) * rng.standard_normal(m.x.shape) * (1 - m.fixed)
    delta = 50.0
    pf = tm.FP64 if prec == "fp64" else tm.FP32_MIXED
    ctx = tm.Context.from_mesh(m, metric=metric, precision=pf)
    ctx.set_restricted_movement(delta, dev(x_init))
    orc = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, metric, delta=delta, x_init=x_init)
    tol_v = RTOL if prec == "fp64" else 1e-5
    x = dev(m.x)
    rc, F, _ = ctx.energy(x)
    assert abs(F - orc.energy(m.x)[1]) <= RTOL * abs(F)
    assert rel(host(ctx.gradient(x)), orc.gradient(m.x)) <= RTOL
    v = rng.standard_normal(m.x.shape)
    yo = orc.hess_apply(m.x, v)
    assert rel(host(ctx.hess_apply(x, dev(v))), yo) <= tol_v
    ctx.linearize(x)
    assert rel(host(ctx.hess_apply_pa(dev(v))), yo) <= tol_v
    if name == "c1":
        xa = dev(m.x)
        r = ctx.newton_solve(xa, max_newton=30)
        assert r.status == tm.OK
        free_ctx = tm.Context.from_mesh(m, metric=metric)
        xb = dev(m.x)
        assert free_ctx.newton_solve(xb, max_newton=30).status == tm.OK
        assert np.linalg.norm(host(xa) - x_init) < np.linalg.norm(host(xb) - x_init)
    ctx.set_restricted_movement(0.0)
    assert abs(ctx.energy(x)[1] - _single(m, metric).energy(m.x)[1]) <= RTOL * F


# ---------------------------------------------------------------- partial assembly
@pytest.mark.parametrize("name,kw,metric", [("c1", dict(nx=5), 2), ("c1", dict(nx=4), 77), ("c2", dict(nx=6), 9),
                                            ("c3", dict(nx=3), 303), ("c3", dict(nx=3), 302), ("c4", dict(nx=2), 303),
                                            ("c3", dict(nx=2, order=4, nq=6), 303)])
def test_partial_assembly_matches_oracle(tm, name, kw, metric):
    m = make(name, 2, **kw)
    scale = 0.3 if metric in (7, 9, 77) else None
    ctx = tm.Context.from_mesh(m, metric=metric, target_scale=scale)
    orc = orc_for(m, metric=metric, W=None if scale is None else np.eye(m.dim) * scale)
    x = dev(m.x)
    ctx.linearize(x)
    for seed in range(2):
        v = np.random.default_rng(seed).standard_normal(m.x.shape)
        y = host(ctx.hess_apply_pa(dev(v)))
        yo = orc.hess_apply(m.x, v)
        assert rel(y, yo) <= RTOL, rel(y, yo)
        assert np.all(y[m.fixed == 1] == 0.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_partial_assembly_general_targets_and_fp32(tm, dim):
    rng = np.random.default_rng(11)
    m = make("c1" if dim == 2 else "c3", 5, nx=3 if dim == 2 else 2)
    Wq = (np.eye(dim) + 0.15 * rng.standard_normal((m.nelem, m.Q, dim, dim))) / 6
    Wq[np.linalg.det(Wq) < 0, :, 0] *= -1
    v = rng.standard_normal(m.x.shape)
    yo = orc_for(m, Wqp=Wq).hess_apply(m.x, v)
    ctx = tm.Context.from_mesh(m, W_per_qp=Wq)
    ctx.linearize(dev(m.x))
    assert rel(host(ctx.hess_apply_pa(dev(v))), yo) <= RTOL
    c32 = tm.Context.from_mesh(m, W_per_qp=Wq, precision=tm.FP32_MIXED)
    c32.linearize(dev(m.x))
    assert rel(host(c32.hess_apply_pa(dev(v))), yo) <= 1e-5


@pytest.mark.parametrize("order,nq,nx,structured", [(1, 2, (3, 3, 2), True), (1, 3, (2, 3, 4), False),
                                                    (2, 3, (3, 2, 1), True),
                                                    (2, 4, (5, 4, 3), False), (3, 4, (4, 3, 2), True),
                                                    (3, 5, (12, 12, 12), True), (3, 5, (7, 5, 3), False),
                                                    (4, 5, (3, 2, 2), False), (4, 6, (3, 3, 3), True)])
def test_fp32_stored_hessian_product_3d(tm, order, nq, nx, structured):
    """The 3D FP32 stored-Hessian product from compact records (mu303, W = I:
    T and the five scaled partials of mu per point) against the oracle's
    FP64 Hessian action, for every order, ragged grids, more elements than
    resident warps, both node-numbering paths, with the boundary fixed. The
    FP32 bound is that of the other FP32 products."""
    m = make("c4", 2, order=order, nq=nq, nx=nx)
    rng = np.random.default_rng(order * 10 + nq)
    v = rng.standard_normal(m.x.shape)
    yo = orc_for(m).hess_apply(m.x, v)
    c32 = tm.Context.from_mesh(m, precision=tm.FP32_MIXED, structured=structured)
    c32.linearize(dev(m.x))
    assert c32.pa_layout()[0] == 14
    y = host(c32.hess_apply_pa(dev(v)))
    assert rel(y, yo) <= 1e-5, rel(y, yo)
    assert np.all(y[m.fixed == 1] == 0.0)
    # the accumulating form: y0 + H v at the free dofs, y0 kept at the fixed ones
    y0 = rng.standard_normal(m.x.shape)
    ya = host(c32.hess_apply_pa(dev(v), out=dev(y0), accumulate=True))
    free = m.fixed == 0
    assert np.all(ya[~free] == y0[~free])
    assert np.abs(ya[free] - (y0[free] + y[free])).max() <= 1e-12 * (np.abs(y0).max() + np.abs(y).max())
    # on FP32 vectors (the FP32 MINRES form): FP32 v, FP32 atomics into y
    v32 = torch.tensor(v, dtype=torch.float32, device="cuda")
    y32 = torch.tensor(np.where(free, 0.0, 7.0), dtype=torch.float32, device="cuda")
    c32.hess_apply_pa_add_f32(v32, y32)
    y32h = y32.cpu().numpy().astype(np.float64)
    assert np.all(y32h[~free] == 7.0)
    assert rel(np.where(free, y32h, 0.0), yo) <= 1e-5


@pytest.mark.parametrize("order,nq,nx,structured,W", [(1, 2, (3, 3, 2), True, False), (2, 3, (3, 2, 3), False, True),
                                                      (3, 5, (7, 5, 3), True, False), (3, 5, (6, 4, 4), False, True),
                                                      (4, 5, (3, 2, 2), True, False), (4, 6, (3, 3, 3), True, True)])
def test_fp32_recomputed_hessian_action_3d(tm, order, nq, nx, structured, W):
    """The 3D FP32 Hessian action recomputed from x (the matrix-free Krylov
    operator of the FP32 forms; compact records built per element in shared
    memory) against the oracle's FP64 Hessian action: every order, ragged
    grids, both node-numbering paths, W = I and a constant non-symmetric W,
    boundary fixed, more elements than resident warps."""
    m = make("c4", 3, order=order, nq=nq, nx=nx)
    okw = {}
    if W:
        Wm = (np.eye(3) + 0.2 * np.random.default_rng(4).standard_normal((3, 3))) / 4
        if np.linalg.det(Wm) < 0:
            Wm[:, 0] *= -1
        m.W = Wm
        okw.update(wkind=oracle.W_CONST, W=Wm)
    orc = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, m.metric, **okw)
    v = np.random.default_rng(order).standard_normal(m.x.shape)
    yo = orc.hess_apply(m.x, v)
    c32 = tm.Context.from_mesh(m, precision=tm.FP32_MIXED, structured=structured)
    y = host(c32.hess_apply(dev(m.x), dev(v)))
    assert rel(y, yo) <= 1e-5, rel(y, yo)
    assert np.all(y[m.fixed == 1] == 0.0)


@pytest.mark.parametrize("case", ["mu14", "mu1", "W", "mu302", "mu98", "composite", "per_point_W", "bulk"])
def test_fp32_compact_and_packed_records_3d(tm, case):
    """Which record a 3D FP32 linearisation stores, and that the product
    from it matches the oracle: compact (14 values) for mu1, mu14, mu303 with
    a constant target (also non-symmetric, and in the FP32-bulk form);
    packed (45) for mu302 and mu98 (not (|T|^2, det T) metrics), for a
    composite metric and for per-point targets."""
    m = make("c3", 4, nx=(3, 2, 2))
    metric = {"mu14": 14, "mu1": 1, "mu302": 302, "mu98": 98}.get(case, 303)
    rng = np.random.default_rng(5)
    okw, ckw = {}, {}
    if case == "W":
        W = (np.eye(3) + 0.2 * rng.standard_normal((3, 3))) / 4
        if np.linalg.det(W) < 0:
            W[:, 0] *= -1
        m.W = W
        okw.update(wkind=oracle.W_CONST, W=W)
    if case == "per_point_W":
        Wq = (np.eye(3) + 0.1 * rng.standard_normal((m.nelem, m.Q, 3, 3))) / 4
        Wq[np.linalg.det(Wq) < 0, :, 0] *= -1
        okw.update(wkind=oracle.W_PER_QP, W=Wq)
        ckw.update(W_per_qp=Wq)
    prec = tm.FP32_BULK if case == "bulk" else tm.FP32_MIXED
    ctx = tm.Context.from_mesh(m, metric=metric, precision=prec, **ckw)
    if case == "composite":
        eta = 0.5 + rng.random((m.nelem, m.Q))
        ctx.set_composite(14, np.eye(3) * 0.3, eta)
        okw.update(metric2=14, W2=np.eye(3) * 0.3, eta2=eta)
    orc = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, metric, **okw)
    ctx.linearize(dev(m.x))
    packed = case in ("mu302", "mu98", "composite", "per_point_W")
    assert ctx.pa_layout() == ((45, 45 * m.Q, 4) if packed else (14, 14 * m.Q + (-14 * m.Q) % 4, 4))
    v = rng.standard_normal(m.x.shape)
    yo = orc.hess_apply(m.x, v)
    assert rel(host(ctx.hess_apply_pa(dev(v))), yo) <= 1e-5


def test_fp32_conversions_round_like_a_cast(tm):
    """The integer-pipe FP64 -> FP32 conversion of the FP32 kernels against
    numpy's IEEE cast (round to nearest even) on random values over the
    whole normal float range, exact ties (both parities), values that round
    up across a binade, the largest finite float and overflow, zeros,
    infinities and NaN; results below 2^-126 become signed zeros. The FP32 ->
    FP64 widening must be exact."""
    rng = np.random.default_rng(17)
    n = 20000
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    f = (sign * (1.0 + rng.random(n)) * 2.0 ** rng.integers(-100, 100, n)).astype(np.float32)   # normal floats
    ulp32 = np.abs(np.spacing(f)).astype(np.float64)
    base = f.astype(np.float64)
    vals = np.concatenate([
        sign * (1.0 + rng.random(n)) * 2.0 ** rng.integers(-100, 100, n),
        base + 0.5 * ulp32 * np.sign(base),          # exact ties
        base + 0.5000001 * ulp32 * np.sign(base),    # just above a tie
        base + 0.4999999 * ulp32 * np.sign(base),    # just below a tie
        np.nextafter(np.float64(1.0), 2.0) * np.array([1.0, -1.0]),
        np.array([2.0 - 2.0 ** -25, 2.0 ** -126, -(2.0 ** -126), 3.4028234663852886e38, 0.0, -0.0]),
    ])
    x = dev(vals)
    f32, back = tm.selftest_convert(x)
    ref = vals.astype(np.float32)
    got = f32.cpu().numpy()
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    assert np.array_equal(back.cpu().numpy(), got.astype(np.float64))
    special = np.array([np.inf, -np.inf, np.nan, 1e39, -1e39, 1e-39, -1e-39, 1e-300])
    f32, back = tm.selftest_convert(dev(special))
    got = f32.cpu().numpy()
    assert got[0] == np.inf and got[1] == -np.inf and np.isnan(got[2])
    assert got[3] == np.inf and got[4] == -np.inf
    assert np.array_equal(got[5:], np.array([0.0, -0.0, 0.0], np.float32)) and np.signbit(got[6])
    b = back.cpu().numpy()
    assert b[0] == np.inf and b[1] == -np.inf and np.isnan(b[2])


def test_inverse_cube_root_within_a_few_ulp(tm):
    """tau^{-1/3} of the FP64 kernels (Newton from an FP32 start) against
    numpy's cube root: within 8 ulp (the reference itself is two roundings)
    over the Newton range, exact cubes,
    the range ends and the library fallback beyond them."""
    rng = np.random.default_rng(9)
    a = np.concatenate([
        10.0 ** rng.uniform(-36, 36, 20000),
        np.array([1.0, 8.0, 27.0, 0.125, 2.0 ** -120, 2.0 ** 120, 2.0 ** -121, 2.0 ** 121, 1e-300, 1e300]),
        (rng.integers(1, 1000, 1000).astype(np.float64)) ** 3,
    ])
    got = host(tm.selftest_rcbrt(dev(a)))
    ref = 1.0 / np.cbrt(a)
    ulp = np.spacing(np.abs(ref))
    assert np.all(np.abs(got - ref) <= 8 * ulp), np.max(np.abs(got - ref) / ulp)


def test_partial_assembly_requires_linearize(tm):
    m = make("c1", 1, nx=2)
    ctx = tm.Context.from_mesh(m)
    with pytest.raises(tm.TmopError):
        ctx.hess_apply_pa(dev(m.x))


# ---------------------------------------------------------------- Jacobi preconditioning
@pytest.mark.parametrize("name,kw,extras", [("c1", dict(nx=4), ""), ("c3", dict(nx=2), ""),
                                            ("c1", dict(nx=3), "composite+delta"), ("c3", dict(nx=2), "fp32"),
                                            ("c3", dict(nx=2), "fp32+W"), ("c3", dict(nx=2), "fp32+composite"),
                                            ("c4", dict(nx=(3, 2, 2)), "fp32"), ("c4", dict(nx=(2, 2, 3)), "fp32+W")])
def test_hessian_diagonal_matches_oracle(tm, name, kw, extras):
    """Diagonal of the partially assembled Hessian against the oracle's
    Hessian action on every unit vector (brute force), 1 at fixed dofs; in
    3D FP32 both from compact records (W = I and a constant non-symmetric W)
    and from packed Hessians (a composite metric)."""
    m = make(name, 5, **kw)
    prec = tm.FP32_MIXED if "fp32" in extras else tm.FP64
    okw = {}
    if "W" in extras.split("+"):
        W = (np.eye(m.dim) + 0.2 * np.random.default_rng(3).standard_normal((m.dim, m.dim))) / 4
        if np.linalg.det(W) < 0:
            W[:, 0] *= -1
        m.W = W
        okw.update(wkind=oracle.W_CONST, W=W)
    ctx = tm.Context.from_mesh(m, precision=prec)
    if "composite" in extras:
        W2 = np.eye(m.dim) * 0.4
        eta = np.full((m.nelem, m.Q), 0.7)
        ctx.set_composite(77 if m.dim == 2 else 14, W2, eta)
        okw.update(metric2=77 if m.dim == 2 else 14, W2=W2, eta2=eta)
    if "delta" in extras:
        ctx.set_restricted_movement(3.0, dev(m.x_ideal))
        okw.update(delta=3.0, x_init=m.x_ideal)
    orc = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, m.metric, **okw)
    x = dev(m.x)
    ctx.linearize(x)
    if prec != tm.FP64 and m.dim == 3:
        assert ctx.pa_layout()[0] == (45 if "composite" in extras else 14)
    d = host(ctx.hessian_diagonal())
    ref = np.ones_like(m.x)
    for a, i in np.argwhere(m.fixed == 0):
        e = np.zeros_like(m.x)
        e[a, i] = 1.0
        ref[a, i] = orc.hess_apply(m.x, e)[a, i]
    tol = RTOL if prec == tm.FP64 else 1e-5
    assert np.abs(d - ref).max() <= tol * np.abs(ref).max()


def test_jacobi_minres_solves_the_same_system(tm):
    m = make("c2", 1, nx=12)
    ctx = tm.Context.from_mesh(m)
    orc = orc_for(m)
    b = orc.gradient(m.x)
    po, _ = orc.minres(m.x, b, rtol=1e-13, maxit=3000)
    p1, it1 = ctx.krylov_solve(dev(m.x), dev(b), krylov_rtol=1e-12, krylov_maxit=3000)
    p2, it2 = ctx.krylov_solve(dev(m.x), dev(b), krylov_rtol=1e-12, krylov_maxit=3000, precond=1)
    assert it1 > 0 and it2 > 0
    assert rel(host(p1), po) <= 1e-9 and rel(host(p2), po) <= 1e-9
    assert it2 < it1


def test_jacobi_newton_converges_with_fewer_iterations(tm):
    m = make("c3", 2, nx=8)
    ctx = tm.Context.from_mesh(m)
    xa, xb = dev(m.x), dev(m.x)
    ra = ctx.newton_solve(xa, max_newton=20)
    rb = ctx.newton_solve(xb, max_newton=20, precond=1)
    assert ra.status == tm.OK and rb.status == tm.OK
    F0 = ctx.energy(dev(m.x))[1]
    assert abs(ra.report["F"] - rb.report["F"]) <= 1e-12 * F0
    assert rb.report["krylov_iterations"] < ra.report["krylov_iterations"]
    assert np.abs(host(xa) - host(xb)).max() < 1e-9 / 16


# ---------------------------------------------------------------- solvers
@pytest.mark.parametrize("krylov", ["minres", "cg"])
def test_krylov_matches_oracle(tm, krylov):
    m = make("c1", 1)
    ctx = tm.Context.from_mesh(m)
    orc = orc_for(m)
    b = orc.gradient(m.x)
    p, it = ctx.krylov_solve(dev(m.x), dev(b), krylov=krylov, krylov_rtol=1e-12, krylov_maxit=1000)
    po, ito = (orc.minres if krylov == "minres" else orc.cg)(m.x, b, rtol=1e-12, maxit=1000)
    assert it > 0 and ito > 0 and abs(it - ito) <= 3
    assert rel(host(p), po) <= 1e-9
    r = orc.hess_apply(m.x, host(p)) - b
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(b)


@pytest.mark.parametrize("delta", [0.0, 2.0])
def test_minres_with_compact_records_solves_the_fp64_system(tm, delta):
    """MINRES with the 3D FP32 compact-record product (which returns v.(Hv)
    itself, so the solver skips its dot pass; with the restricted-movement
    term it does not, and the separate pass runs): the solution of H p = b
    against the oracle's FP64 Hessian, to the FP32 operator's accuracy, and
    against the oracle's MINRES solution."""
    m = make("c3", 2, nx=(4, 3, 3))
    okw = dict(delta=delta, x_init=m.x_ideal) if delta else {}
    orc = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, m.metric, **okw)
    ctx = tm.Context.from_mesh(m, precision=tm.FP32_MIXED)
    if delta:
        ctx.set_restricted_movement(delta, dev(m.x_ideal))
    b = orc.gradient(m.x)
    p, it = ctx.krylov_solve(dev(m.x), dev(b), krylov_rtol=1e-9, krylov_maxit=3000)
    assert it > 0
    r = orc.hess_apply(m.x, host(p)) - b
    assert np.linalg.norm(r) <= 1e-4 * np.linalg.norm(b), np.linalg.norm(r) / np.linalg.norm(b)
    po, _ = orc.minres(m.x, b, rtol=1e-12, maxit=3000)
    assert rel(host(p), po) <= 1e-3


@pytest.mark.parametrize("precond", [0, 1, 2])
def test_fp32_krylov_vectors_solve_the_same_system(tm, precond):
    """The FP32 forms run MINRES on FP32 vectors by default (krylov_fp64 = 0):
    the solution matches the FP64-vector solve of the same FP32 operator and
    the oracle's FP64 system to the FP32 operator's accuracy, in about the
    same number of iterations, for plain, Jacobi and two-level MINRES."""
    m = make("c4", 2, nx=(6, 5, 4))
    orc = orc_for(m)
    b = orc.gradient(m.x)
    ctx = tm.Context.from_mesh(m, precision=tm.FP32_MIXED)
    p32, it32 = ctx.krylov_solve(dev(m.x), dev(b), krylov_rtol=1e-6, krylov_maxit=3000, precond=precond)
    p64, it64 = ctx.krylov_solve(dev(m.x), dev(b), krylov_rtol=1e-6, krylov_maxit=3000, precond=precond,
                                 krylov_fp64=1)
    assert it32 > 0 and it64 > 0 and abs(it32 - it64) <= max(3, it64 // 10), (it32, it64)
    assert rel(host(p32), host(p64)) <= 1e-4
    r = orc.hess_apply(m.x, host(p32)) - b
    assert np.linalg.norm(r) <= 1e-4 * np.linalg.norm(b), np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("metric,scale", [(2, None), (7, 1.0 / 8)])
def test_newton_matches_oracle_history(tm, metric, scale):
    """Section 3.4 Newton on 8x8 order-2: the same accepted step lengths and
    F history as the oracle while F is above rounding level (F > 1e-8 F0;
    below that the acceptance tests compare rounding noise, F* = 0 here), then
    convergence to the uniform grid (F* = 0) with det A > 0 throughout."""
    m = make("c1", 1)
    ctx = tm.Context.from_mesh(m, metric=metric, target_scale=scale)
    orc = orc_for(m, metric=metric, W=None if scale is None else np.eye(2) * scale)
    rco, xo, hist = orc.newton(m.x, max_newton=20)
    F0 = hist[0, 0]
    x = dev(m.x)
    assert abs(ctx.energy(x)[1] - F0) <= RTOL * F0
    compared = 0
    for it in range(len(hist) - 1):
        if hist[it, 0] <= 1e-8 * F0:
            break
        r = ctx.newton_step(x, max_newton=20)
        assert r.status == tm.OK and r.report["min_detA"] > 0
        assert r.report["alpha"] == hist[it + 1, 3]
        Fk, Fo = r.report["F"], hist[it + 1, 0]
        assert abs(Fk - Fo) <= 1e-9 * Fo + 1e-12 * F0, (it, Fk, Fo)
        compared += 1
    assert compared >= 3
    x2 = dev(m.x)
    res = ctx.newton_solve(x2, max_newton=20)
    assert res.status == tm.OK and res.report["F"] <= 1e-12 * F0 and res.report["min_detA"] > 0
    assert np.abs(host(x2) - m.x_ideal).max() < 1e-11
    # the matrix-free Krylov operator converges to the same mesh
    x3 = dev(m.x)
    res3 = ctx.newton_solve(x3, max_newton=20, matrix_free=1)
    assert res3.status == tm.OK
    assert np.abs(host(x3) - host(x2)).max() < 1e-11


def test_newton_strict_monotone_and_barrier(tm):
    m = make("c2", 2, nx=16)
    ctx = tm.Context.from_mesh(m)
    x = dev(m.x)
    F = [ctx.energy(x)[1]]
    for _ in range(6):
        r = ctx.newton_step(x, f_factor=1.0)
        if r.status != tm.OK:
            break
        F.append(r.report["F"])
        assert r.report["min_detA"] > 0
    assert len(F) >= 4 and np.all(np.diff(F) < 0)


def test_linesearch_exhaustion_reports_status(tm):
    """With max_halvings = 0 and an impossible acceptance factor the step is
    rejected: status LINESEARCH, x unchanged (Section 3.4 termination)."""
    m = make("c1", 1, nx=4)
    ctx = tm.Context.from_mesh(m)
    x = dev(m.x)
    r = ctx.newton_step(x, max_halvings=1, f_factor=1e-30)
    assert r.status == tm.ERR_LINESEARCH
    assert np.array_equal(host(x), m.x)


# ---------------------------------------------------------------- FP32 forms
def test_fp32_bulk_bounds(tm):
    """FP32 element arithmetic everywhere, FP64 reductions. Coordinates are
    shifted to the element's first node in FP64 before rounding, so A carries
    relative error ~eps32 k. Measured bounds (stated in the design notes):
    F 1e-6, gradient 1e-5, Hessian action 1e-5 (normwise, against the FP64
    oracle)."""
    for name, kw in [("c2", {}), ("c3", dict(nx=12))]:
        m = make(name, 1, **kw)
        ctx = tm.Context.from_mesh(m, precision=tm.FP32_BULK)
        check_all(tm, m, ctx, orc_for(m), rtol_F=1e-6, rtol_vec=1e-5)


def test_fp32_mixed_is_fp64_except_hessian_action(tm):
    m = make("c3", 1, nx=12)
    ctx = tm.Context.from_mesh(m, precision=tm.FP32_MIXED)
    orc = orc_for(m)
    x = dev(m.x)
    rc, F, md = ctx.energy(x)
    _, Fo, mdo = orc.energy(m.x)
    assert abs(F - Fo) <= RTOL * Fo and abs(md - mdo) <= RTOL * abs(mdo)
    assert rel(host(ctx.gradient(x)), orc.gradient(m.x)) <= RTOL
    v = np.random.default_rng(1).standard_normal(m.x.shape)
    assert rel(host(ctx.hess_apply(x, dev(v))), orc.hess_apply(m.x, v)) <= 1e-5


def test_fp32_mixed_newton_reaches_fp64_solution(tm):
    """FP32 Hessian action inside MINRES, FP64 gradient and line search: the
    Newton iterates converge to the same mesh as plain FP64 (F within 1e-10
    relative), det A > 0 throughout."""
    m = make("c3", 3, nx=8)
    x64, x32 = dev(m.x), dev(m.x)
    c64 = tm.Context.from_mesh(m)
    F0 = c64.energy(x64)[1]
    r64 = c64.newton_solve(x64, max_newton=20)
    r32 = tm.Context.from_mesh(m, precision=tm.FP32_MIXED).newton_solve(x32, max_newton=30)
    assert r64.status == tm.OK and r32.status == tm.OK
    F64, F32 = r64.report["F"], r32.report["F"]
    # F* > 0 here (sheared cube); compare against the initial F (no ill-posed ratio)
    assert abs(F32 - F64) <= 1e-10 * F0
    assert np.abs(host(x32) - host(x64)).max() <= 1e-8 / 16
    assert r32.report["min_detA"] > 0


@pytest.mark.gpu
def test_fma_peak_is_measured_and_plausible(tm):
    """The roofline denominators of the ALU-bound kernels: tmop_fma_peak
    measures FP64 and FP32 multiply-add throughput on this GPU. Each is
    positive and no higher than the unit-count bound at the 2.07 GHz maximum
    clock of a GB300-class part (152 SMs; 2 FP64 and 128 FP32 FMA per SM and
    clock), and FP32 runs far faster than FP64 on this part."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    g64, ms64 = tm.fma_peak(tm.PEAK_FP64)
    g32, _ = tm.fma_peak(tm.PEAK_FP32)
    g32x2, _ = tm.fma_peak(tm.PEAK_FP32X2)
    assert ms64 > 0.1
    assert 0 < g64 <= sms * 2.2 * 2 * 2 * 1.02
    assert 0 < max(g32, g32x2) <= sms * 2.2 * 128 * 2 * 1.02
    assert max(g32, g32x2) > 8 * g64
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    import ctypes as C
    g = C.c_double(0.0)
    assert tm.load().tmop_fma_peak(tm.PEAK_FP64, C.c_void_p(small.data_ptr()), 16, C.byref(g), None, None) == tm.ERR_CAPACITY
    assert tm.load().tmop_fma_peak(7, C.c_void_p(small.data_ptr()), 16, C.byref(g), None, None) == tm.ERR_ARG


# ---------------------------------------------------------------- two-level preconditioner
@pytest.mark.parametrize("name,kw,prec", [("c5", dict(nx=6), "fp64"), ("c4", dict(nx=4), "fp64"),
                                          ("c4", dict(nx=(4, 3, 5)), "fp32"), ("c3", dict(nx=(3, 4, 3)), "fp64")])
def test_twolevel_coarse_part_matches_oracle(tm, name, kw, prec):
    """The coarse part of the two-level preconditioner, P (alpha K_c)^-1 P^t r
    (tmop_precond_apply with precond 2 minus precond 1, i.e. minus the
    Jacobi part), and alpha against the oracle's dense definition
    (oracle/twolevel.py) with the oracle's Hessian: FP64 to 1e-10, the FP32
    form (FP32 Hessian action and transforms) to 1e-5."""
    from oracle import twolevel as otl
    m = make(name, 3, **kw)
    ctx = tm.Context.from_mesh(m, precision=tm.FP64 if prec == "fp64" else tm.FP32_MIXED)
    orc = orc_for(m)
    x = dev(m.x)
    r = np.random.default_rng(4).standard_normal(m.x.shape) * (1 - m.fixed)
    z2, a_gpu = ctx.precond_apply(x, dev(r), 2)
    z1, a1 = ctx.precond_apply(x, dev(r), 1)
    assert a1 == 0.0 and a_gpu > 0
    a_ref = otl.alpha(lambda v: orc.hess_apply(m.x, v), m.nx, m.order, m.dim)
    tol = 1e-10 if prec == "fp64" else 1e-5
    assert abs(a_gpu - a_ref) <= tol * a_ref, (a_gpu, a_ref)
    ref = otl.coarse_part(r, m.nx, m.order, a_ref)
    assert rel(host(z2) - host(z1), ref) <= tol


def test_twolevel_minres_solves_the_same_system_in_fewer_iterations(tm):
    """MINRES with the two-level preconditioner returns the oracle's MINRES
    solution of H p = g (1e-9) in well under half the iterations of plain
    MINRES and of Jacobi (3D order 3, 6^3 hexes, mu303)."""
    m = make("c4", 2, nx=6)
    ctx = tm.Context.from_mesh(m)
    orc = orc_for(m)
    b = orc.gradient(m.x)
    po, _ = orc.minres(m.x, b, rtol=1e-13, maxit=3000)
    p0, it0 = ctx.krylov_solve(dev(m.x), dev(b), krylov_rtol=1e-12, krylov_maxit=3000)
    p1, it1 = ctx.krylov_solve(dev(m.x), dev(b), krylov_rtol=1e-12, krylov_maxit=3000, precond=1)
    p2, it2 = ctx.krylov_solve(dev(m.x), dev(b), krylov_rtol=1e-12, krylov_maxit=3000, precond=2)
    assert it0 > 0 and it1 > 0 and it2 > 0
    for p in (p0, p1, p2):
        assert rel(host(p), po) <= 1e-9
    assert 2 * it2 < min(it0, it1), (it0, it1, it2)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_twolevel_newton_reaches_the_same_mesh(tm, prec):
    """Newton with the two-level preconditioner (3D order 3, 8^3 hexes,
    mu303) stops at the same F and nodes as with plain MINRES, with under
    half the MINRES iterations."""
    m = make("c4", 1, nx=8)
    ctx = tm.Context.from_mesh(m, precision=tm.FP64 if prec == "fp64" else tm.FP32_MIXED)
    xa, xb = dev(m.x), dev(m.x)
    ra = ctx.newton_solve(xa, max_newton=20)
    rb = ctx.newton_solve(xb, max_newton=20, precond=2)
    assert ra.status == tm.OK and rb.status == tm.OK
    F0 = ctx.energy(dev(m.x))[1]
    assert abs(ra.report["F"] - rb.report["F"]) <= 1e-12 * F0
    assert 2 * rb.report["krylov_iterations"] < ra.report["krylov_iterations"], (ra.report, rb.report)
    assert np.abs(host(xa) - host(xb)).max() < 1e-9 / 24


def test_twolevel_needs_a_boundary_fixed_structured_grid(tm):
    """Tangential relaxation frees boundary dofs, which the coarse space does
    not have: the two-level form is refused (TMOP_ERR_ARG), Jacobi is not."""
    m = mg.make_mesh("c1", 1, tangential=True)
    ctx = tm.Context.from_mesh(m)
    x = dev(m.x)
    r = dev(np.ones_like(m.x) * (1 - m.fixed))
    ctx.precond_apply(x, r, 1)
    with pytest.raises(tm.TmopError):
        ctx.precond_apply(x, r, 2)
    with pytest.raises(tm.TmopError):
        ctx.krylov_solve(x, r, precond=2)


# ---------------------------------------------------------------- deterministic (colour-ordered) scatter
@pytest.mark.parametrize("name,kw,prec,structured,delta", [
    ("c3", dict(nx=(4, 3, 5)), "fp64", True, 0.0), ("c3", dict(nx=(3, 4, 3)), "fp64", False, 1.5),
    ("c4", dict(nx=4), "fp32", True, 0.0), ("c2", dict(nx=(7, 6)), "fp64", False, 0.0),
    ("c2", dict(nx=(5, 8)), "fp32", True, 2.0)])
def test_deterministic_scatter(tm, name, kw, prec, structured, delta):
    """Colour-ordered sums (tmop_set_deterministic): the gradient, the
    recomputed and the stored-Hessian products and the Jacobi diagonal are
    bitwise equal on two calls, agree with the atomic sums to 1e-13
    normwise, and match the oracle (gradient, products: 1e-12 in FP64, 1e-5
    for the FP32 Hessian action). Structured grids use the 2^d parity
    colours, unstructured ones the greedy colouring; with and without the
    restricted-movement term."""
    m = make(name, 4, **kw)
    pf = tm.FP64 if prec == "fp64" else tm.FP32_MIXED
    okw = dict(delta=delta, x_init=m.x_ideal) if delta else {}
    orc = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, m.metric, **okw)
    ca = tm.Context.from_mesh(m, precision=pf, structured=structured)
    cd = tm.Context.from_mesh(m, precision=pf, structured=structured)
    if delta:
        for c in (ca, cd):
            c.set_restricted_movement(delta, dev(m.x_ideal))
    cd.set_deterministic(True)
    x = dev(m.x)
    v = np.random.default_rng(8).standard_normal(m.x.shape)
    vd = dev(v)
    tolv = RTOL if prec == "fp64" else 1e-5

    def outs(c):
        c.linearize(x)
        return {"g": host(c.gradient(x)), "hv": host(c.hess_apply(x, vd)), "pa": host(c.hess_apply_pa(vd)),
                "diag": host(c.hessian_diagonal())}
    d1, d2, a1 = outs(cd), outs(cd), outs(ca)
    for k in d1:
        assert np.array_equal(d1[k], d2[k]), k
        assert rel(d1[k], a1[k]) <= 1e-13, (k, rel(d1[k], a1[k]))
    assert rel(d1["g"], orc.gradient(m.x)) <= RTOL
    ref = orc.hess_apply(m.x, v)
    assert rel(d1["hv"], ref) <= tolv and rel(d1["pa"], ref) <= tolv


@pytest.mark.parametrize("prec,precond", [("fp64", 0), ("fp32", 0), ("fp32", 2)])
def test_deterministic_newton_is_bitwise_reproducible(tm, prec, precond):
    """With colour-ordered sums two Newton solves from the same mesh give the
    same iterate bit for bit (MINRES, line search and all), and the same
    mesh as the atomic sums to rounding."""
    m = make("c4", 2, nx=5)
    pf = tm.FP64 if prec == "fp64" else tm.FP32_MIXED
    cd = tm.Context.from_mesh(m, precision=pf)
    cd.set_deterministic(True)
    xs, reps = [], []
    for _ in range(2):
        xx = dev(m.x)
        r = cd.newton_solve(xx, max_newton=20, precond=precond)
        assert r.status == tm.OK
        xs.append(host(xx))
        reps.append(r.report)
    assert np.array_equal(xs[0], xs[1])
    assert reps[0]["krylov_iterations"] == reps[1]["krylov_iterations"] and reps[0]["F"] == reps[1]["F"]
    ca = tm.Context.from_mesh(m, precision=pf)
    xa = dev(m.x)
    ra = ca.newton_solve(xa, max_newton=20, precond=precond)
    assert ra.status == tm.OK
    F0 = ca.energy(dev(m.x))[1]
    assert abs(ra.report["F"] - reps[0]["F"]) <= 1e-12 * F0
    assert np.abs(host(xa) - xs[0]).max() < 1e-9 / 15


# ---------------------------------------------------------------- stacks of equal 2D grids
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_grid_stack_matches_the_union_and_the_oracle(tm, prec):
    """Three 2D grids stacked as one structured problem (structured[2] = 3,
    the nodes of one grid after another) give the energy, gradient and
    Hessian actions of the same meshes as one unstructured union, and of the
    oracle on each grid; Newton with the two-level preconditioner (one coarse
    vertex grid per grid) reaches the union's plain-MINRES F."""
    from paper_1807_09807_gb300 import learned as L
    ms = [make("c5", 20 + i, nx=(5, 4)) for i in range(3)]
    pf = tm.FP64 if prec == "fp64" else tm.FP32_MIXED
    cs, xh = L.union_context(ms, pf)
    assert cs.stacked
    en = np.concatenate([m.elem_nodes + i * ms[0].nnode for i, m in enumerate(ms)]).astype(np.int32)
    fx = np.concatenate([m.fixed for m in ms], axis=1)
    cu = tm.Context(2, 3, xh.shape[1], en, fx, ms[0].nq, ms[0].metric, precision=pf)
    x = dev(xh)
    v = np.random.default_rng(6).standard_normal(xh.shape)
    tol = RTOL if prec == "fp64" else 1e-5
    _, Fs, mds = cs.energy(x)
    _, Fu, mdu = cu.energy(x)
    assert abs(Fs - Fu) <= 1e-13 * Fu and mds == mdu
    gs, gu = host(cs.gradient(x)), host(cu.gradient(x))
    assert rel(gs, gu) <= 1e-13
    hs, hu = host(cs.hess_apply(x, dev(v))), host(cu.hess_apply(x, dev(v)))
    assert rel(hs, hu) <= (1e-13 if prec == "fp64" else 1e-6)
    N = ms[0].nnode
    for i, m in enumerate(ms):
        orc = orc_for(m)
        assert rel(gs[:, i * N:(i + 1) * N], orc.gradient(m.x)) <= RTOL
        assert rel(hs[:, i * N:(i + 1) * N], orc.hess_apply(m.x, v[:, i * N:(i + 1) * N])) <= tol
    xa, xb = dev(xh), dev(xh)
    ra = cu.newton_solve(xa, max_newton=20)
    rb = cs.newton_solve(xb, max_newton=20, precond=2)
    assert ra.status == tm.OK and rb.status == tm.OK
    assert abs(ra.report["F"] - rb.report["F"]) <= 1e-12 * Fu
    assert rb.report["krylov_iterations"] < ra.report["krylov_iterations"]
