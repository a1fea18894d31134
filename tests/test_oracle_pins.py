"""Pins of the CPU oracle against what the paper and the mathematics fix,
independently of the oracle's own code: textbook quadrature rules (numpy),
interpolation identities, the literal metric definitions (numpy.linalg),
invariances, finite differences, closed forms on affine meshes, the exact
area identity, the textbook Q_k stiffness matrix and brute-force Newton
convergence."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1807_09807_gb300 import meshgen as mg

rng = np.random.default_rng(12345)


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 6, 8])
def test_gauss_legendre_matches_numpy_and_is_exact(q):
    pts, wts = oracle.gauss_legendre(q)
    t, w = np.polynomial.legendre.leggauss(q)   # library rule on [-1, 1]
    np.testing.assert_allclose(pts, 0.5 * (t + 1.0), rtol=0, atol=1e-15)
    np.testing.assert_allclose(wts, 0.5 * w, rtol=0, atol=1e-15)
    assert abs(wts.sum() - 1.0) < 1e-15
    for deg in range(2 * q):                       # exact through degree 2q-1
        assert abs(np.dot(wts, pts ** deg) - 1.0 / (deg + 1)) < 1e-14


@pytest.mark.parametrize("q", [2, 3, 4, 5, 6, 7])
def test_gauss_lobatto_is_exact_and_has_textbook_nodes(q):
    pts, wts = oracle.gauss_lobatto(q)
    assert pts[0] == 0.0 and pts[-1] == 1.0
    for deg in range(2 * q - 2):                   # exact through degree 2q-3
        assert abs(np.dot(wts, pts ** deg) - 1.0 / (deg + 1)) < 1e-14
    # not exact at degree 2q-2 (a Lobatto rule, not a Gauss rule)
    assert abs(np.dot(wts, pts ** (2 * q - 2)) - 1.0 / (2 * q - 1)) > 1e-8
    # interior nodes: roots of P'_{q-1} (numpy Legendre derivative roots)
    if q > 2:
        r = np.sort(np.polynomial.legendre.Legendre.basis(q - 1).deriv().roots())
        np.testing.assert_allclose(pts[1:-1], 0.5 * (r + 1.0), atol=1e-14)


def test_gll_golden_values():
    """Closed-form Gauss-Lobatto nodes and weights (tests/golden/gll_closed_forms.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.txt")
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        q, rest = line.split(":")
        nodes, weights = rest.split("|")
        nodes = [float(eval(s, {"sqrt": np.sqrt})) for s in nodes.split(",")]
        weights = [float(eval(s, {"sqrt": np.sqrt})) for s in weights.split(",")]
        pts, wts = oracle.gauss_lobatto(int(q))
        np.testing.assert_allclose(pts, 0.5 * (np.array(nodes) + 1), atol=1e-15)
        np.testing.assert_allclose(wts, 0.5 * np.array(weights), atol=1e-15)


# ---------------------------------------------------------------- basis
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_lagrange_basis(k):
    nodes, _ = oracle.gauss_lobatto(k + 1)
    for xi in [0.0, 0.13, 0.5, 0.77, 1.0]:
        phi, dphi = oracle.lagrange(nodes, xi)
        assert abs(phi.sum() - 1.0) < 1e-14          # partition of unity
        assert abs(dphi.sum()) < 1e-12
        # library: numpy polynomial through (nodes, e_i)
        for i in range(k + 1):
            c = np.polynomial.polynomial.polyfit(nodes, np.eye(k + 1)[i], k)
            assert abs(np.polynomial.polynomial.polyval(xi, c) - phi[i]) < 1e-11
            dc = np.polynomial.polynomial.polyder(c)
            assert abs(np.polynomial.polynomial.polyval(xi, dc) - dphi[i]) < 1e-9
    for j, xj in enumerate(nodes):                   # interpolation property
        phi, _ = oracle.lagrange(nodes, xj)
        np.testing.assert_allclose(phi, np.eye(k + 1)[j], atol=1e-14)


# ---------------------------------------------------------------- metrics
METRICS_2D = [1, 2, 7, 9, 14, 77, 98]
METRICS_3D = [1, 14, 98, 302, 303]


def _definition(mid, T):
    """Literal definitions of Table 3.1 / Section 3.2 with numpy.linalg."""
    d = T.shape[0]
    tau = np.linalg.det(T)
    n2 = np.sum(T * T)
    Tinv = np.linalg.inv(T)
    I = np.eye(d)
    return {
        1: n2,
        2: n2 / (2 * tau) - 1,
        7: np.sum((T - Tinv.T) ** 2),
        9: tau * np.sum((T - Tinv.T) ** 2),
        14: np.sum((T - I) ** 2),
        77: 0.5 * (tau - 1 / tau) ** 2,
        98: np.sum((T - I) ** 2) / tau,
        302: n2 * np.sum(Tinv ** 2) / 9 - 1,
        303: n2 / (3 * np.cbrt(tau) ** 2) - 1,
    }[mid]


def _rand_T(d):
    while True:
        T = np.eye(d) + 0.4 * rng.standard_normal((d, d))
        if np.linalg.det(T) > 0.2:
            return T


def _rot(d):
    Qm, _ = np.linalg.qr(rng.standard_normal((d, d)))
    if np.linalg.det(Qm) < 0:
        Qm[:, 0] *= -1
    return Qm


@pytest.mark.parametrize("d,mid", [(2, m) for m in METRICS_2D] + [(3, m) for m in METRICS_3D])
def test_metric_value_matches_definition(d, mid):
    for _ in range(20):
        T = _rand_T(d)
        rc, mu, _, _ = oracle.metric(mid, T)
        assert rc == 0
        assert abs(mu - _definition(mid, T)) < 1e-12 * max(1.0, abs(mu))


@pytest.mark.parametrize("d,mid", [(2, m) for m in METRICS_2D] + [(3, m) for m in METRICS_3D])
def test_metric_derivatives_against_central_fd(d, mid):
    for _ in range(5):
        T = _rand_T(d)
        dT = rng.standard_normal((d, d))
        rc, mu, P, dP = oracle.metric(mid, T, dT)
        h = 1e-6
        Pfd = np.zeros((d, d))
        for i in range(d):
            for j in range(d):
                E = np.zeros((d, d)); E[i, j] = h
                Pfd[i, j] = (_definition(mid, T + E) - _definition(mid, T - E)) / (2 * h)
        np.testing.assert_allclose(P, Pfd, rtol=1e-7, atol=1e-7 * np.abs(P).max())
        _, _, Pp, _ = oracle.metric(mid, T + h * dT)
        _, _, Pm, _ = oracle.metric(mid, T - h * dT)
        np.testing.assert_allclose(dP, (Pp - Pm) / (2 * h), rtol=1e-6, atol=1e-7 * np.abs(dP).max())


@pytest.mark.parametrize("d,mid", [(2, 2), (2, 7), (2, 9), (2, 14), (2, 77), (2, 98), (3, 14), (3, 98), (3, 302),
                                   (3, 303)])
def test_metric_zero_at_identity(d, mid):
    rc, mu, P, _ = oracle.metric(mid, np.eye(d))
    assert abs(mu) < 1e-15 and np.abs(P).max() < 1e-15


@pytest.mark.parametrize("d,mid,scale_inv", [(2, 1, False), (2, 2, True), (2, 7, False), (2, 9, False),
                                             (2, 77, False), (3, 1, False), (3, 302, True), (3, 303, True)])
def test_metric_invariances(d, mid, scale_inv):
    for _ in range(10):
        T = _rand_T(d)
        mu = oracle.metric(mid, T)[1]
        R = _rot(d)
        assert abs(oracle.metric(mid, R @ T)[1] - mu) < 1e-12 * max(1, abs(mu))
        if scale_inv:
            assert abs(oracle.metric(mid, 2.7 * T)[1] - mu) < 1e-12 * max(1, abs(mu))


def test_barrier_metrics_reject_inverted():
    T = np.array([[1.0, 0.0], [0.0, -0.5]])
    for mid in (2, 7, 9, 77, 98):
        assert oracle.metric(mid, T)[0] == oracle.ERR_INVERTED
    T3 = np.diag([1.0, 1.0, -1.0])
    for mid in (98, 302, 303):
        assert oracle.metric(mid, T3)[0] == oracle.ERR_INVERTED


@pytest.mark.parametrize("d", [2, 3])
def test_mu98_closed_forms(d):
    """mu98 (Section 4.3.2) on T = s I is d (s - 1)^2 / s^d; it is not
    rotation invariant: on a rotation R by angle t (2D) it is |R - I|^2 =
    2 d_rot (1 - cos t) with det R = 1."""
    for s_ in (0.5, 1.0, 1.7):
        mu = oracle.metric(98, s_ * np.eye(d))[1]
        assert abs(mu - d * (s_ - 1) ** 2 / s_ ** d) < 1e-14
    t = 0.3
    R = np.eye(d)
    R[:2, :2] = [[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]]
    assert abs(oracle.metric(98, R)[1] - 4 * (1 - np.cos(t))) < 1e-14


# ---------------------------------------------------------------- mesh level
def _problem(m, metric=None, W=None):
    wk = oracle.W_IDENTITY if W is None else oracle.W_CONST
    return oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq,
                          metric or m.metric, quad_kind=m.quad_kind, wkind=wk, W=W)


def _small(name, **kw):
    base = dict(c1=dict(), c2=dict(nx=6), c3=dict(nx=3), c4=dict(nx=2), c5=dict(nx=4))[name]
    base.update(kw)
    return mg.make_mesh(name, 1, **base)


@pytest.mark.parametrize("name", ["c1", "c2", "c3", "c4"])
def test_sum_of_w_detA_is_volume(name):
    """det A is a polynomial the Gauss rule integrates exactly, so
    sum_E sum_q w_q det A = |Omega| (= 1: the sine and shear maps keep volume)."""
    m = _small(name)
    p = _problem(m)
    w, _ = p.tables()
    J = p.jacobians(m.x)
    vol = np.sum(np.linalg.det(J) * w[None, :])
    assert abs(vol - 1.0) < 1e-13


@pytest.mark.parametrize("dim,order,nq", [(2, 2, 4), (2, 3, 5), (3, 2, 4), (3, 3, 5)])
def test_affine_mesh_closed_forms(dim, order, nq):
    """Global affine map M on the uniform grid: A = M / n_x at every point;
    shape metrics give F = N_E mu(M); the gradient vanishes at free dofs."""
    nx = 3
    x0, en, fixed = mg.structured(dim, order, nx)
    M = np.eye(dim) + 0.3 * rng.standard_normal((dim, dim))
    if np.linalg.det(M) < 0:
        M[:, 0] *= -1
    x = M @ x0
    mid = 2 if dim == 2 else 303
    p = oracle.Problem(dim, order, en, x.shape[1], fixed, nq, mid)
    J = p.jacobians(x)
    np.testing.assert_allclose(J, np.broadcast_to(M / nx, J.shape), atol=1e-14)
    rc, F, md = p.energy(x)
    assert rc == 0
    assert abs(F - en.shape[0] * _definition(mid, M)) < 1e-12 * max(1, F)
    assert abs(md - np.linalg.det(M / nx)) < 1e-14
    g = p.gradient(x)
    assert np.abs(g).max() < 1e-13 * max(1.0, F)


def test_mu2_shear_closed_form():
    """mu2 of the shear [[1,s],[0,1]] is s^2/2, so F = N_E s^2 / 2."""
    x0, en, fixed = mg.structured(2, 2, 5)
    s = 0.37
    x = np.array([[1, s], [0, 1]]) @ x0
    p = oracle.Problem(2, 2, en, x.shape[1], fixed, 4, 2)
    assert abs(p.energy(x)[1] - 25 * s * s / 2) < 1e-13


def test_mu7_equal_size_target_zero_on_ideal_mesh():
    """With the equal-size target W2 = sqrt(|Omega|/N_E) I (eq. (3.1)), T = I on
    the uniform grid, so mu7 and its gradient vanish."""
    m = mg.make_mesh("c2", 1, nx=6)
    p = _problem(m, metric=7, W=np.eye(2) / 6)
    x0, _, _ = mg.structured(2, 3, 6)   # the plain grid (c2's x_ideal carries the sine map)
    rc, F, _ = p.energy(x0)
    assert rc == 0 and abs(F) < 1e-13 and np.abs(p.gradient(x0)).max() < 1e-13
    rc, F, _ = p.energy(m.x_ideal)
    assert rc == 0 and F > 1e-3


def test_inverted_mesh_gives_infinite_energy():
    m = _small("c1")
    x = m.x_ideal.copy()
    # fold one interior node across its neighbours
    node = m.elem_nodes[27, 4]
    x[0, node] += 0.2
    p = _problem(m)
    rc, F, md = p.energy(x)
    assert rc == oracle.ERR_INVERTED and F == np.inf and md <= 0


@pytest.mark.parametrize("name,metric", [("c1", 2), ("c1", 7), ("c1", 9), ("c1", 77), ("c2", 2),
                                         ("c3", 303), ("c3", 302), ("c4", 303)])
def test_gradient_against_central_fd(name, metric):
    m = _small(name, nx=2) if name != "c1" else _small(name, nx=3)
    p = _problem(m, metric=metric, W=(np.eye(m.dim) / 3 if metric in (7, 9, 77) else None))
    g = p.gradient(m.x)
    free = np.argwhere(m.fixed == 0)
    sel = free[rng.choice(len(free), size=min(25, len(free)), replace=False)]
    h = 1e-6
    for a, i in sel:
        xp = m.x.copy(); xp[a, i] += h
        xm = m.x.copy(); xm[a, i] -= h
        fd = (p.energy(xp)[1] - p.energy(xm)[1]) / (2 * h)
        assert abs(fd - g[a, i]) < 1e-6 * max(1.0, np.abs(g).max())
    assert np.all(g[m.fixed == 1] == 0.0)


@pytest.mark.parametrize("name,metric", [("c1", 2), ("c1", 7), ("c1", 77), ("c3", 303), ("c3", 302)])
def test_hessian_action_fd_and_symmetry(name, metric):
    m = _small(name, nx=2) if name != "c1" else _small(name, nx=3)
    p = _problem(m, metric=metric, W=(np.eye(m.dim) / 3 if metric in (7, 77) else None))
    free = 1 - m.fixed
    v = rng.standard_normal(m.x.shape) * free
    u = rng.standard_normal(m.x.shape) * free
    Hv = p.hess_apply(m.x, v)
    Hu = p.hess_apply(m.x, u)
    h = 1e-6
    fd = (p.gradient(m.x + h * v) - p.gradient(m.x - h * v)) / (2 * h)
    assert np.linalg.norm(Hv - fd) < 1e-6 * np.linalg.norm(Hv)
    assert abs(np.vdot(u, Hv) - np.vdot(v, Hu)) < 1e-12 * np.linalg.norm(Hv) * np.linalg.norm(u)
    assert np.all(Hv[m.fixed == 1] == 0.0)
    # masked input: fixed entries of v are ignored
    vb = v + 5.0 * m.fixed
    np.testing.assert_array_equal(p.hess_apply(m.x, vb), Hv)


def _textbook_stiffness(dim, order, nx):
    """Reference-element Q_k stiffness K_ij = int grad phi_i . grad phi_j
    assembled over the grid, built from exact 1D polynomial integrals
    (numpy polynomials, no quadrature) and Kronecker products."""
    nodes, _ = oracle.gauss_lobatto(order + 1)
    n = order + 1
    polys = [np.polynomial.Polynomial.fit(nodes, np.eye(n)[i], order).convert() for i in range(n)]
    M1 = np.zeros((n, n)); K1 = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            M1[i, j] = (polys[i] * polys[j]).integ()(1.0) - (polys[i] * polys[j]).integ()(0.0)
            dd = polys[i].deriv() * polys[j].deriv()
            K1[i, j] = dd.integ()(1.0) - dd.integ()(0.0)
    if dim == 2:   # local index = j*n + i (x fastest) -> kron(y-part, x-part)
        Ke = np.kron(M1, K1) + np.kron(K1, M1)
    else:
        Ke = np.kron(np.kron(M1, M1), K1) + np.kron(np.kron(M1, K1), M1) + np.kron(np.kron(K1, M1), M1)
    x0, en, fixed = mg.structured(dim, order, nx)
    N = x0.shape[1]
    K = np.zeros((N, N))
    for e in range(en.shape[0]):
        idx = en[e]
        K[np.ix_(idx, idx)] += Ke
    return K, x0, en, fixed


@pytest.mark.parametrize("dim,order,nq", [(2, 2, 4), (2, 3, 5), (3, 2, 4)])
def test_mu14_hessian_is_twice_textbook_stiffness(dim, order, nq):
    nx = 3 if dim == 2 else 2
    K, x0, en, fixed = _textbook_stiffness(dim, order, nx)
    N = x0.shape[1]
    p = oracle.Problem(dim, order, en, N, fixed, nq, 14)
    xr = x0 + 0.01 * rng.standard_normal(x0.shape) * (1 - fixed)
    v = rng.standard_normal(x0.shape) * (1 - fixed)
    y = p.hess_apply(xr, v)
    ref = 2.0 * (K @ v.T).T * (1 - fixed)
    assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max()


def test_mu14_one_newton_step_is_exact():
    """mu14 with W = I is quadratic in x: one Newton step reaches the discrete
    harmonic map, which is the uniform grid for the unit-square boundary."""
    m = _small("c1", nx=4)
    p = _problem(m, metric=14)
    rc, x, hist = p.newton(m.x, max_newton=3, krylov="cg", krylov_rtol=1e-14)
    assert np.abs(x - m.x_ideal).max() < 1e-12
    assert hist[1, 3] == 1.0            # full step accepted


def test_minres_and_cg_solve_the_hessian_system():
    m = _small("c1", nx=3)
    p = _problem(m)
    b = p.gradient(m.x)
    for solver in (p.minres, p.cg):
        s, it = solver(m.x, b, rtol=1e-12, maxit=500)
        assert it > 0
        r = p.hess_apply(m.x, s) - b
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("metric,W", [(2, None), (7, "W2")])
def test_newton_converges_to_uniform_grid(metric, W):
    """With the boundary fixed on the unit square, mu2 (and mu7 with the
    equal-size target) is minimised by the uniform grid (F* = 0)."""
    m = mg.make_mesh("c1", 1)
    Wm = np.eye(2) / 8 if W == "W2" else None
    p = _problem(m, metric=metric, W=Wm)
    rc, x, hist = p.newton(m.x, max_newton=20)
    F0 = hist[0, 0]
    assert rc in (oracle.OK, oracle.ERR_LINESEARCH, oracle.ERR_NOT_CONVERGED)
    assert rc == oracle.OK
    # F* = 0; what is left is the rounding of mu2 = |T|^2/(2 tau) - 1 near T = I
    assert hist[-1, 0] <= 1e-14 * F0
    assert np.abs(x - m.x_ideal).max() < 1e-12
    assert np.all(hist[:, 2] > 0)                       # det A > 0 at every iterate
    # quadratic convergence at the end: |g| drops faster than linearly
    g = hist[:, 1]
    k = np.argmax(g < 1e-3 * g[0])
    assert g[k + 1] < g[k] ** 1.5 / g[0] ** 0.5 or g[k + 1] <= 1e-12 * g[0]


def test_newton_strict_decrease_is_monotone():
    m = mg.make_mesh("c1", 2)
    p = _problem(m)
    rc, x, hist = p.newton(m.x, max_newton=8, f_factor=1.0)
    F = hist[:, 0]
    assert np.all(np.diff(F) < 0)


def _general_W(d, nelem=None, Q=None):
    W = np.eye(d) + 0.3 * rng.standard_normal((d, d))
    if np.linalg.det(W) < 0:
        W[:, 0] *= -1
    if nelem is None:
        return W
    Ws = np.eye(d) + 0.2 * rng.standard_normal((nelem, Q, d, d))
    Ws[np.linalg.det(Ws) < 0, :, 0] *= -1
    return Ws


@pytest.mark.parametrize("dim,mid", [(2, 2), (2, 7), (3, 303), (3, 302)])
def test_general_constant_target_closed_form_and_fd(dim, mid):
    """Non-symmetric constant W: on an affine mesh T = (M / n_x) W^-1 and
    F = N_E det W mu(T); gradient and Hessian action match central FD."""
    nx = 2
    order, nq = (2, 4)
    x0, en, fixed = mg.structured(dim, order, nx)
    M = np.eye(dim) + 0.2 * rng.standard_normal((dim, dim))
    W = _general_W(dim) / nx
    p = oracle.Problem(dim, order, en, x0.shape[1], fixed, nq, mid, wkind=oracle.W_CONST, W=W)
    x = M @ x0
    T = (M / nx) @ np.linalg.inv(W)
    rc, F, _ = p.energy(x)
    assert abs(F - en.shape[0] * np.linalg.det(W) * _definition(mid, T)) < 1e-12 * max(1, abs(F))
    xj = x + 0.02 / nx * rng.standard_normal(x.shape) * (1 - fixed)
    g = p.gradient(xj)
    h = 1e-6
    free = np.argwhere(fixed == 0)
    for a, i in free[rng.choice(len(free), size=min(12, len(free)), replace=False)]:
        xp = xj.copy(); xp[a, i] += h
        xm = xj.copy(); xm[a, i] -= h
        fd = (p.energy(xp)[1] - p.energy(xm)[1]) / (2 * h)
        assert abs(fd - g[a, i]) < 1e-6 * np.abs(g).max()
    v = rng.standard_normal(x.shape) * (1 - fixed)
    Hv = p.hess_apply(xj, v)
    fdH = (p.gradient(xj + h * v) - p.gradient(xj - h * v)) / (2 * h)
    assert np.linalg.norm(Hv - fdH) < 1e-6 * np.linalg.norm(Hv)


@pytest.mark.parametrize("dim,mid", [(2, 2), (3, 303)])
def test_per_point_target_fd(dim, mid):
    """Targets given at every quadrature point (Section 3.1)."""
    nx, order, nq = 2, 2, 4
    x0, en, fixed = mg.structured(dim, order, nx)
    Q = nq ** dim
    Ws = _general_W(dim, en.shape[0], Q) / nx
    p = oracle.Problem(dim, order, en, x0.shape[1], fixed, nq, mid, wkind=oracle.W_PER_QP, W=Ws)
    xj = x0 + 0.02 / nx * rng.standard_normal(x0.shape) * (1 - fixed)
    # energy against the definition, point by point from the oracle's own A
    pi = oracle.Problem(dim, order, en, x0.shape[1], fixed, nq, mid)
    w, _ = pi.tables()
    J = pi.jacobians(xj)
    Fdef = sum(w[q] * np.linalg.det(Ws[e, q]) * _definition(mid, J[e, q] @ np.linalg.inv(Ws[e, q]))
               for e in range(en.shape[0]) for q in range(Q))
    assert abs(p.energy(xj)[1] - Fdef) < 1e-12 * abs(Fdef)
    g = p.gradient(xj)
    h = 1e-6
    free = np.argwhere(fixed == 0)
    for a, i in free[rng.choice(len(free), size=min(12, len(free)), replace=False)]:
        xp = xj.copy(); xp[a, i] += h
        xm = xj.copy(); xm[a, i] -= h
        assert abs((p.energy(xp)[1] - p.energy(xm)[1]) / (2 * h) - g[a, i]) < 1e-6 * np.abs(g).max()


def test_curved_boundary_optimum_is_not_the_initial_lattice():
    """The curved-boundary workload of the learned proposal: with the top
    boundary on y = 1 + 0.15 sin(pi x) and every boundary node fixed, mu2
    Newton converges to a mesh that differs from both the mapped lattice and
    its jittered copy, so a proposal has more to predict than the jitter."""
    m = mg.make_mesh("c5curved", 3, nx=4, order=2, nq=4)
    top = m.fixed[1] == 1
    on_curve = np.isclose(m.x[1], 1.0 + 0.15 * np.sin(np.pi * m.x[0])) & (m.x[1] > 1.0 - 1e-12)
    assert np.any(on_curve) and np.all(m.fixed[:, on_curve] == 1) and np.any(top)
    p = _problem(m)
    rc, x, hist = p.newton(m.x, max_newton=30)
    assert rc == oracle.OK and hist[-1, 1] <= 1e-12 * hist[0, 1]
    assert np.abs(x - m.x_ideal).max() > 1e-3
    assert np.array_equal(x[m.fixed == 1], m.x[m.fixed == 1])


def test_tangential_relaxation_on_axis_parallel_boundaries():
    """Section 4.1: boundary nodes slide along axis-parallel faces (only the
    normal displacement is fixed). Boundary nodes stay on their faces exactly,
    the gradient matches FD on the sliding dofs, and Newton still reaches the
    uniform grid (F* = 0)."""
    m = mg.make_mesh("c1", 3, nx=4, tangential=True)
    p = _problem(m)
    x0 = m.x
    on_face = m.fixed == 1
    assert np.array_equal(x0[on_face], m.x_ideal[on_face])           # normal coordinates untouched
    slide = (m.fixed == 0) & (np.abs(x0 - m.x_ideal) > 0)
    g = p.gradient(x0)
    h = 1e-6
    for a, i in np.argwhere(slide)[:10]:
        xp = x0.copy(); xp[a, i] += h
        xm = x0.copy(); xm[a, i] -= h
        assert abs((p.energy(xp)[1] - p.energy(xm)[1]) / (2 * h) - g[a, i]) < 1e-6 * np.abs(g).max()
    rc, x, hist = p.newton(x0, max_newton=20)
    assert rc == oracle.OK
    assert np.array_equal(x[on_face], x0[on_face])
    assert np.abs(x - m.x_ideal).max() < 1e-11


@pytest.mark.parametrize("dim,ma,mb", [(2, 1, 77), (2, 2, 7), (3, 303, 14)])
def test_composite_metric(dim, ma, mb):
    """Section 4.2, eq. (4.1): mu = mu_a(A W^-1) + eta_q mu_b(A W2^-1), with
    point weights eta (the paper's ICF example combines mu1/W1 with
    eta(r) mu77/W2). F against the literal sum evaluated with numpy.linalg at
    the oracle's own Jacobians; gradient and Hessian action against FD."""
    m = mg.make_mesh("c1" if dim == 2 else "c3", 2, nx=3 if dim == 2 else 2)
    W2 = (np.eye(dim) + 0.2 * rng.standard_normal((dim, dim))) * (0.7 / 3)   # non-symmetric
    if np.linalg.det(W2) < 0:
        W2[:, 0] *= -1
    eta = 0.5 + rng.random((m.nelem, m.Q))
    p = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, ma, metric2=mb, W2=W2, eta2=eta)
    pa = _problem(m, metric=ma)
    w, _ = pa.tables()
    J = pa.jacobians(m.x)
    W2i = np.linalg.inv(W2)
    Fdef = sum(w[q] * (_definition(ma, J[e, q]) + np.linalg.det(W2) * eta[e, q] * _definition(mb, J[e, q] @ W2i))
               for e in range(m.nelem) for q in range(m.Q))
    rc, F, _ = p.energy(m.x)
    assert rc == 0 and abs(F - Fdef) < 1e-12 * abs(Fdef)
    g = p.gradient(m.x)
    h = 1e-6
    free = np.argwhere(m.fixed == 0)
    for a, i in free[rng.choice(len(free), size=min(12, len(free)), replace=False)]:
        xp = m.x.copy(); xp[a, i] += h
        xm = m.x.copy(); xm[a, i] -= h
        assert abs((p.energy(xp)[1] - p.energy(xm)[1]) / (2 * h) - g[a, i]) < 1e-6 * np.abs(g).max()
    v = rng.standard_normal(m.x.shape) * (1 - m.fixed)
    Hv = p.hess_apply(m.x, v)
    fd = (p.gradient(m.x + h * v) - p.gradient(m.x - h * v)) / (2 * h)
    assert np.linalg.norm(Hv - fd) < 1e-6 * np.linalg.norm(Hv)


@pytest.mark.parametrize("dim", [2, 3])
def test_replication_metric_keeps_the_initial_mesh(dim):
    """Section 4.3.2: with the per-point target W0 = A(x_init), mu98(A W0^-1)
    = |T0 - I|^2 / det T0 vanishes exactly at x_init and is positive
    elsewhere, so x_init is the minimiser: F = 0 and g = 0 there, and Newton
    from a perturbed mesh goes back to it."""
    m = mg.make_mesh("c1" if dim == 2 else "c3", 1, nx=4 if dim == 2 else 2)
    A0 = _problem(m).jacobians(m.x)
    p = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, 98, wkind=oracle.W_PER_QP, W=A0)
    rc, F, _ = p.energy(m.x)
    assert rc == 0 and abs(F) < 1e-13
    assert np.abs(p.gradient(m.x)).max() < 1e-12
    x1 = m.x + 0.05 / (m.order * 4) * rng.uniform(-1, 1, m.x.shape) * (1 - m.fixed)
    assert p.energy(x1)[1] > 1e-6
    rc, x, hist = p.newton(x1, max_newton=20)
    assert rc == 0 and np.abs(x - m.x).max() < 1e-10, (rc, np.abs(x - m.x).max(), hist[:, 0])


def test_gamma_blend_restricts_movement():
    """Section 4.3.2 second restricted-movement algorithm: mu' = (1 - gamma)
    mu98(A W0^-1) + gamma mu2(A), W0 = A(x_init). Written as eq. (4.1) with
    mu98 first and eta2 = gamma / (1 - gamma) (the same objective times
    1 / (1 - gamma), so the same minimiser). The optimised mesh moves further
    from x_init as gamma grows, and the unrestricted (mu2 alone) optimum moves
    furthest."""
    m = mg.make_mesh("c1", 1, nx=4)
    A0 = _problem(m).jacobians(m.x)
    moved = []
    for gamma in (0.05, 0.3, 0.7):
        eta = np.full((m.nelem, m.Q), gamma / (1 - gamma))
        p = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, 98, wkind=oracle.W_PER_QP,
                           W=A0, metric2=2, eta2=eta)
        rc, x, _ = p.newton(m.x, max_newton=30)
        assert rc == 0
        moved.append(np.linalg.norm(x - m.x))
    rc, x, _ = _problem(m, metric=2).newton(m.x, max_newton=30)
    assert rc == 0
    moved.append(np.linalg.norm(x - m.x))
    assert moved[0] > 0 and all(a < b for a, b in zip(moved, moved[1:])), moved


def _textbook_mass(dim, order, nx):
    """Reference-element Q_k mass matrix M_ij = int phi_i phi_j assembled over
    the grid (exact 1D polynomial integrals, Kronecker products)."""
    nodes, _ = oracle.gauss_lobatto(order + 1)
    n = order + 1
    polys = [np.polynomial.Polynomial.fit(nodes, np.eye(n)[i], order).convert() for i in range(n)]
    M1 = np.array([[((polys[i] * polys[j]).integ()(1.0) - (polys[i] * polys[j]).integ()(0.0)) for j in range(n)]
                   for i in range(n)])
    Me = np.kron(M1, M1) if dim == 2 else np.kron(np.kron(M1, M1), M1)
    _, en, _ = mg.structured(dim, order, nx)
    N = en.max() + 1
    M = np.zeros((N, N))
    for e in range(en.shape[0]):
        M[np.ix_(en[e], en[e])] += Me
    return M


def test_restricted_movement_closed_forms():
    """Section 4.3.1, eq. (4.2): adds sum_E int delta |x - x_init|^2 dx_t.
    (i) a rigid translation c of a free mesh adds delta |c|^2 N_E (the metric
    part is translation invariant); (ii) with mu14 the Hessian is
    2 (K + delta M) with the textbook stiffness K and mass M; (iii) FD."""
    delta = 3.7
    for dim, order, nq, nx in [(2, 2, 4, 3), (3, 2, 4, 2)]:
        x0, en, fixed = mg.structured(dim, order, nx)
        xi = x0 + 0.01 / nx * rng.standard_normal(x0.shape)
        mid = 2 if dim == 2 else 303
        p0 = oracle.Problem(dim, order, en, x0.shape[1], None, nq, mid)
        pd = oracle.Problem(dim, order, en, x0.shape[1], None, nq, mid, delta=delta, x_init=xi)
        c = rng.standard_normal((dim, 1)) * 0.05
        F0 = p0.energy(xi)[1]
        Fd = pd.energy(xi + c)[1]
        assert abs(Fd - F0 - delta * np.sum(c * c) * en.shape[0]) < 1e-12 * max(1.0, Fd)
        # (ii) mu14
        K, _, _, _ = _textbook_stiffness(dim, order, nx)
        M = _textbook_mass(dim, order, nx)
        p14 = oracle.Problem(dim, order, en, x0.shape[1], fixed, nq, 14, delta=delta, x_init=xi)
        v = rng.standard_normal(x0.shape) * (1 - fixed)
        y = p14.hess_apply(xi, v)
        ref = 2.0 * ((K + delta * M) @ v.T).T * (1 - fixed)
        assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max()
        # (iii) gradient and Hessian action against FD
        pf = oracle.Problem(dim, order, en, x0.shape[1], fixed, nq, mid, delta=delta, x_init=xi)
        x = xi + 0.02 / nx * rng.standard_normal(x0.shape) * (1 - fixed)
        g = pf.gradient(x)
        h = 1e-6
        free = np.argwhere(fixed == 0)
        for a, i in free[rng.choice(len(free), size=min(10, len(free)), replace=False)]:
            xp = x.copy(); xp[a, i] += h
            xm = x.copy(); xm[a, i] -= h
            assert abs((pf.energy(xp)[1] - pf.energy(xm)[1]) / (2 * h) - g[a, i]) < 1e-6 * np.abs(g).max()
        Hv = pf.hess_apply(x, v)
        fd = (pf.gradient(x + h * v) - pf.gradient(x - h * v)) / (2 * h)
        assert np.linalg.norm(Hv - fd) < 1e-6 * np.linalg.norm(Hv)


def test_restricted_movement_scaled_target_and_masking():
    """The penalty is integrated over the target element (weights w_q det W):
    with W = s I a rigid translation adds delta |c|^2 N_E s^d; and fixed
    entries of a Hessian-action direction are ignored by the penalty too."""
    dim, order, nq, nx, s, delta = 2, 3, 5, 3, 0.4, 2.5
    x0, en, fixed = mg.structured(dim, order, nx)
    xi = x0 + 0.01 / nx * rng.standard_normal(x0.shape)
    W = np.eye(dim) * s
    p0 = oracle.Problem(dim, order, en, x0.shape[1], None, nq, 2, wkind=oracle.W_CONST, W=W)
    pd = oracle.Problem(dim, order, en, x0.shape[1], None, nq, 2, wkind=oracle.W_CONST, W=W, delta=delta, x_init=xi)
    c = np.array([[0.03], [-0.02]])
    assert abs(pd.energy(xi + c)[1] - p0.energy(xi)[1] - delta * np.sum(c * c) * en.shape[0] * s ** dim) < 1e-12
    pf = oracle.Problem(dim, order, en, x0.shape[1], fixed, nq, 2, delta=delta, x_init=xi)
    v = rng.standard_normal(x0.shape)
    np.testing.assert_array_equal(pf.hess_apply(xi, v), pf.hess_apply(xi, v * (1 - fixed)))


# ---------------------------------------------------------------- two-level preconditioner (reference)
from oracle import twolevel as otl  # noqa: E402


@pytest.mark.parametrize("ns,k", [((3, 4), 3), ((3, 3, 2), 2), ((2, 3), 1)])
def test_twolevel_interpolation_is_the_product_of_hat_functions(ns, k):
    """Column v of P is the vertex hat function prod_a max(0, 1 - |n_a X_a - v_a|)
    evaluated at the lattice points X = (e + z_i) / n (z: GLL nodes): the
    textbook formula, not the (1 - z, z) construction of the reference."""
    z, _ = oracle.gauss_lobatto(k + 1)
    P = otl.interpolation(ns, k)
    dim = len(ns)
    coords = []
    for n in ns:
        c = np.array([(e + z[i]) / n for e in range(n) for i in range(k)] + [1.0])
        coords.append(c)
    grids = np.meshgrid(*coords, indexing="ij")          # [x][y][z] axes
    pts = np.stack([g.transpose(tuple(reversed(range(dim)))).reshape(-1) for g in grids])  # x fastest
    vs = list(itertools.product(*[range(1, n) for n in reversed(ns)]))
    for col, v in enumerate(vs):
        v = v[::-1]
        hat = np.ones(pts.shape[1])
        for a in range(dim):
            hat *= np.maximum(0.0, 1.0 - np.abs(ns[a] * pts[a] - v[a]))
        assert np.abs(P[:, col] - hat).max() < 1e-13


@pytest.mark.parametrize("ns", [(3, 4), (3, 2, 3)])
def test_twolevel_coarse_laplacian_is_half_the_order1_mu14_hessian(ns):
    """K_c equals half the oracle's mu14 Hessian of the order-1 vertex grid
    (mu14 = |T - I|^2 with W = I is quadratic: its Hessian is twice the
    reference-space Q1 stiffness), on the interior vertices."""
    dim = len(ns)
    x0, en, fixed = mg.structured(dim, 1, ns)
    N = x0.shape[1]
    p = oracle.Problem(dim, 1, en, N, fixed, 2, 14)
    interior = np.where(fixed[0] == 0)[0]
    H = np.zeros((len(interior), len(interior)))
    for j, node in enumerate(interior):
        e = np.zeros_like(x0)
        e[0, node] = 1.0
        H[:, j] = p.hess_apply(x0, e)[0, interior]
    assert np.abs(otl.coarse_laplacian(ns) - 0.5 * H).max() < 1e-13


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 3), (3, 2)])
def test_twolevel_alpha_is_two_for_mu14(dim, k):
    """For mu14 the Hessian is twice the order-k stiffness, whose energy of a
    Q1 vertex field (which Q_k contains) is its Q1 energy: alpha = 2 exactly."""
    ns = (3, 4) if dim == 2 else (2, 3, 3)
    x0, en, fixed = mg.structured(dim, k, ns)
    p = oracle.Problem(dim, k, en, x0.shape[1], fixed, k + 2, 14)
    a = otl.alpha(lambda v: p.hess_apply(x0, v), ns, k, dim)
    assert abs(a - 2.0) < 1e-12


def test_twolevel_apply_is_symmetric_positive_definite():
    """M^-1 as a matrix (2D, order 2, 3 x 4 elements, a positive diagonal):
    symmetric and positive definite, as MINRES needs."""
    ns, k = (3, 4), 2
    Lf = [k * n + 1 for n in ns]
    N = Lf[0] * Lf[1]
    dinv = np.random.default_rng(7).uniform(0.5, 2.0, (2, N))
    M = np.zeros((2 * N, 2 * N))
    for j in range(2 * N):
        e = np.zeros((2, N))
        e.reshape(-1)[j] = 1.0
        M[:, j] = otl.apply(e, dinv, ns, k, 1.7).reshape(-1)
    assert np.abs(M - M.T).max() < 1e-13
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0
