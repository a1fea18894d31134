"""Learned initial iterate: the MLP kernels against the FP64 reference MLP
(oracle/mlp.py), the patch kernels against an independent numpy
construction, and the gain of the trained proposal over plain Newton."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_1807_09807_gb300 import meshgen as mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1807_09807_gb300 import build as cuda_build
    cuda_build.build()
    from paper_1807_09807_gb300 import learned
    learned.lib()
    return learned


def bf16_bits(a):
    """float array -> bfloat16 bit patterns (as int16) and their float64 values."""
    r = omlp.bf16_round(a)
    bits = (r.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16).view(np.int16)
    return bits, r


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("batch", [64, 192, 1024])
def test_mlp_gradients_match_reference(L, batch):
    rng = np.random.default_rng(batch)
    net = L.MLP(200, 18, 256, seed=5)
    flat = rng.standard_normal(net.num_params).astype(np.float32) * 0.08
    net.set(flat)
    params = net.unflatten(net.get(0))
    Xf = rng.standard_normal((batch, 200))
    bits, Xr = bf16_bits(Xf)
    Xd = torch.zeros((batch, net.ld), dtype=torch.int16, device="cuda")
    Xd[:, :200] = torch.tensor(bits, device="cuda")
    T = rng.standard_normal((batch, 18)).astype(np.float32)
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    net.gradients(Xd, torch.tensor(T, device="cuda"), loss)
    g = net.unflatten(net.get(1))
    Lo, go = omlp.backward(Xr, T.astype(np.float64), params, bf16=True)
    assert abs(loss.item() - Lo) <= 1e-5 * Lo
    for k, (a, b) in enumerate(zip(g, go)):
        assert _rel(a, b) <= 3e-3, (k, _rel(a, b))
    Y = net.forward(Xd)[:, :18].cpu().numpy()
    Yo, _ = omlp.forward(Xr, params, bf16=True)
    assert _rel(Y, Yo) <= 1e-3


def test_mlp_adam_training_fits_a_smooth_map(L):
    """Adam on a small regression (targets a fixed random linear map of the
    inputs, through tanh): the loss falls by well over an order of magnitude."""
    rng = np.random.default_rng(0)
    net = L.MLP(64, 8, 128, seed=1)
    S = 8192
    Xf = rng.standard_normal((S, 64))
    bits, Xr = bf16_bits(Xf)
    M = rng.standard_normal((64, 8)) / 8
    T = np.tanh(Xr @ M).astype(np.float32)
    Xd = torch.zeros((S, net.ld), dtype=torch.int16, device="cuda")
    Xd[:, :64] = torch.tensor(bits, device="cuda")
    Td = torch.tensor(T, device="cuda")
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    first = None
    for it in range(300):
        sl = slice((it % 8) * 1024, (it % 8 + 1) * 1024)
        net.gradients(Xd[sl], Td[sl], loss)
        if first is None:
            first = loss.item()
        net.adam(2e-3)
    assert loss.item() < first / 20


def test_mlp_adam_step_matches_the_update_rule(L):
    """Two Adam steps on every parameter block (W1, b1, W2, b2, W3, b3) against
    the update written out in numpy float32: m = 0.9 m + 0.1 g,
    v = 0.999 v + 0.001 g^2, w -= lr (m / (1 - 0.9^t)) / (sqrt(v / (1 - 0.999^t)) + 1e-8)."""
    rng = np.random.default_rng(3)
    net = L.MLP(40, 6, 64, seed=2)
    B = 256
    bits, Xr = bf16_bits(rng.standard_normal((B, 40)))
    Xd = torch.zeros((B, net.ld), dtype=torch.int16, device="cuda")
    Xd[:, :40] = torch.tensor(bits, device="cuda")
    Td = torch.tensor(rng.standard_normal((B, 6)).astype(np.float32), device="cuda")
    w = net.get(0).astype(np.float32)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    for t, lr in ((1, np.float32(1e-3)), (2, np.float32(5e-4))):
        net.gradients(Xd, Td)
        g = net.get(1).astype(np.float32)
        net.adam(float(lr))
        m = np.float32(0.9) * m + np.float32(0.1) * g
        v = np.float32(0.999) * v + np.float32(0.001) * g * g
        mh = m / (np.float32(1) - np.float32(0.9) ** t)
        vh = v / (np.float32(1) - np.float32(0.999) ** t)
        w = w - lr * mh / (np.sqrt(vh) + np.float32(1e-8))
        got = net.get(0)
        assert np.allclose(got, w, rtol=1e-5, atol=1e-7), np.abs(got - w).max()
    # the next forward pass uses the updated weights (their bf16 copies)
    Y = net.forward(Xd)[:, :6].cpu().numpy()
    Yo, _ = omlp.forward(Xr, net.unflatten(w), bf16=True)
    assert _rel(Y, Yo) <= 1e-3


def _features_numpy(m, x, ex, ey):
    k, Nx, Ny = m.order, m.nx[0] * m.order + 1, m.nx[1] * m.order + 1
    P = x.reshape(2, Ny, Nx)

    def qx(gx, gy):
        if gx < 0:
            return 2 * P[:, gy, 0] - P[:, gy, -gx]
        if gx > Nx - 1:
            return 2 * P[:, gy, Nx - 1] - P[:, gy, 2 * (Nx - 1) - gx]
        return P[:, gy, gx]

    def pos(gx, gy):
        if gy < 0:
            return 2 * qx(gx, 0) - qx(gx, -gy)
        if gy > Ny - 1:
            return 2 * qx(gx, Ny - 1) - qx(gx, 2 * (Ny - 1) - gy)
        return qx(gx, gy)

    c = 0.25 * (P[:, k * ey, k * ex] + P[:, k * ey, k * ex + k] + P[:, k * ey + k, k * ex] + P[:, k * ey + k, k * ex + k])
    side = 3 * k + 1
    xi, _ = oracle.gauss_lobatto(k + 1)           # uniform reference lattice inside an element
    ref = [np.floor(a / k) - 1 + xi[a % k] - 0.5 for a in range(side)]
    f = np.zeros(2 * side * side)
    for b in range(side):
        for a in range(side):
            p = pos(k * (ex - 1) + a, k * (ey - 1) + b)
            f[2 * (b * side + a):2 * (b * side + a) + 2] = (p - c) * m.nx[0] - np.array([ref[a], ref[b]])
    return f


def test_patch_features_targets_apply(L):
    m = mg.make_mesh("c5", 7, nx=(5, 4))
    x0 = torch.tensor(m.x, device="cuda")
    X = L.features(m, x0, 256).cpu().numpy()
    for e in range(m.nelem):
        ref = _features_numpy(m, m.x, e % 5, e // 5)
        got = X[e, :len(ref)].astype(np.int16).view(np.uint16).astype(np.uint32) << 16
        got = got.view(np.float32).astype(np.float64)
        bits, r = bf16_bits(ref)
        np.testing.assert_array_equal(got, r)
        assert np.all(X[e, len(ref):] == 0)
    x1 = m.x + 1e-3 * np.random.default_rng(0).standard_normal(m.x.shape) * (1 - m.fixed)
    T = L.targets(m, x0, torch.tensor(x1, device="cuda"))
    Y = torch.zeros((m.nelem, 64), dtype=torch.float32, device="cuda")
    Y[:, :T.shape[1]] = T
    xp = L.apply(m, x0, torch.tensor(m.fixed, device="cuda"), Y).cpu().numpy()
    # every free node off the right/top boundary is owned by exactly one element
    assert np.abs(xp - x1).max() <= 1e-9
    assert np.array_equal(xp[m.fixed == 1], m.x[m.fixed == 1])
    # a damped proposal moves each owned free node by the same fraction
    xh = L.apply(m, x0, torch.tensor(m.fixed, device="cuda"), Y, scale=0.25).cpu().numpy()
    assert np.abs(xh - (m.x + 0.25 * (x1 - m.x))).max() <= 1e-9


def test_concurrent_data_generation_matches_sequential(L):
    """Chunks solved by four host threads on their own streams give the
    samples of the one-thread run, in the same order: features bitwise, the
    Newton-converged targets within the solver tolerance, every chunk
    converged."""
    from paper_1807_09807_gb300 import tmop as tm
    a = L.make_dataset(n_meshes=12, seed0=1000, nx=16, chunk=2, workers=4)
    b = L.make_dataset(n_meshes=12, seed0=1000, nx=16, chunk=2, workers=1)
    assert len(a.newton) == len(b.newton) == 6 and all(s == tm.OK for s, _, _ in a.newton + b.newton)
    assert torch.equal(a.X, b.X)
    Ta, Tb = a.T.double(), b.T.double()
    assert float((Ta - Tb).abs().max()) <= 1e-6 * float(Tb.abs().max())
    # with the coarse stage (each thread solves the vertex grids in its own coarse context)
    a = L.make_dataset(n_meshes=8, seed0=1000, nx=16, chunk=2, preset="c5curved", coarse=True, workers=4)
    b = L.make_dataset(n_meshes=8, seed0=1000, nx=16, chunk=2, preset="c5curved", coarse=True, workers=1)
    assert all(s == tm.OK for s, _, _ in a.newton + b.newton)
    assert a.X.shape == b.X.shape and a.T.shape == b.T.shape   # features of the coarse-stage mesh (FP64 atomics)
    Ta, Tb = a.T.double(), b.T.double()
    assert float((Ta - Tb).abs().max()) <= 1e-5 * float(Tb.abs().max())


def test_learned_proposal_gain(L):
    """Train on Newton-converged displacements of 256 seeded 32x32 order-3
    meshes (mu2, jitter 0.15h), apply to unseen 64x64 meshes: the proposal is
    valid, lowers F, and Newton from it needs fewer Newton and MINRES
    iterations than from the jittered mesh, to the same final F."""
    from paper_1807_09807_gb300 import tmop as tm
    ds = L.make_dataset(n_meshes=256, seed0=1000, chunk=128)
    assert all(s == tm.OK for s, _, _ in ds.newton)
    net = L.MLP(L.n_features(3), L.n_targets(3), 256, seed=0)
    hist = L.train(net, ds, epochs=12, batch=2048, lr=2e-3)
    print("training loss per epoch:", ["%.3e" % h for h in hist])
    zero_loss = float((ds.T.double() ** 2).sum(dim=1).mean())     # predicting no displacement
    assert hist[-1] < 0.02 * zero_loss
    gains = []
    for seed in (5000, 5001):
        m = mg.make_mesh("c5apply", seed, nx=64)
        ctx = tm.Context.from_mesh(m, precision=tm.FP32_MIXED)
        x0 = torch.tensor(m.x, device="cuda")
        fx = torch.tensor(m.fixed, device="cuda")
        prop = L.propose(net, m, ctx, x0, fx)
        assert prop.used and prop.F < 0.5 * prop.F0 and prop.min_detA > 0
        xa, xb = x0.clone(), prop.x.clone()
        # the same absolute target for both starts: 1e-10 |g(x0)|
        g0 = torch.linalg.norm(ctx.gradient(x0)).item()
        ra = ctx.newton_solve(xa, max_newton=30, rtol=1e-30, atol=1e-10 * g0)
        rb = ctx.newton_solve(xb, max_newton=30, rtol=1e-30, atol=1e-10 * g0)
        assert ra.status == tm.OK and rb.status == tm.OK
        assert abs(ra.report["F"] - rb.report["F"]) <= 1e-6 * prop.F0
        assert rb.report["min_detA"] > 0
        assert rb.report["krylov_iterations"] < ra.report["krylov_iterations"]
        gains.append((ra.report["iterations"], rb.report["iterations"], ra.report["krylov_iterations"],
                      rb.report["krylov_iterations"]))
    print("newton/krylov without vs with proposal:", gains)


def test_lattice_vertices_and_prolongation(L):
    """The coarse stage's transfers: the vertex gather is the lattice nodes
    (k i, k j); the prolongation of a bilinear vertex field a + bX + cY + dXY
    reproduces it exactly at every lattice node (X, Y) = ((e + z_i) / n_x,
    (f + z_j) / n_y) (z: Gauss-Lobatto nodes), adds it to x_in at the free
    dofs and leaves the fixed ones alone."""
    m = mg.make_mesh("c5curved", 3, nx=(5, 4))
    k, (nx, ny) = m.order, m.nx
    Nx, Ny, Nv = k * nx + 1, k * ny + 1, (nx + 1) * (ny + 1)
    x = torch.tensor(m.x, device="cuda")
    xv = torch.empty((2, Nv + 3), dtype=torch.float64, device="cuda")   # a padded vertex stride
    L.lattice_vertices(m, x, m.nnode, xv, Nv + 3)
    ref = m.x.reshape(2, Ny, Nx)[:, ::k, ::k].reshape(2, -1)
    assert np.array_equal(xv[:, :Nv].cpu().numpy(), ref)
    coef = [(0.3, -0.2, 0.5, 0.7), (-0.1, 0.4, 0.2, -0.6)]
    vi, vj = np.meshgrid(np.arange(nx + 1) / nx, np.arange(ny + 1) / ny)
    f = np.stack([a + b * vi + c * vj + d * vi * vj for a, b, c, d in coef]).reshape(2, -1)
    xv1 = xv.clone()
    xv1[:, :Nv] += torch.tensor(f, device="cuda")
    out = torch.empty_like(x)
    fx = torch.tensor(m.fixed, device="cuda")
    L.lattice_prolong_add(m, xv, xv1, Nv + 3, x, fx, m.nnode, out)
    z, _ = oracle.gauss_lobatto(k + 1)
    X = np.array([(min(g // k, nx - 1) + z[g - k * min(g // k, nx - 1)]) / nx for g in range(Nx)])
    Y = np.array([(min(g // k, ny - 1) + z[g - k * min(g // k, ny - 1)]) / ny for g in range(Ny)])
    GX, GY = np.meshgrid(X, Y)
    fref = np.stack([a + b * GX + c * GY + d * GX * GY for a, b, c, d in coef]).reshape(2, -1)
    exp = m.x + fref * (1 - m.fixed)
    assert np.abs(out.cpu().numpy() - exp).max() < 1e-14


def test_coarse_stage_proposal_gain_on_curved_boundary(L):
    """The curved top boundary moves the optimum ~6 h away from the mapped
    lattice, which a 3x3-element patch cannot see. With the coarse stage (the
    element-vertex problem solved by Newton and interpolated), a network
    trained on 128 seeded 32x32 curved meshes proposes a valid start with
    lower F on unseen curved meshes, and Newton (FP32 form) from it reaches
    the same F as from the jittered mesh in fewer MINRES iterations."""
    from paper_1807_09807_gb300 import tmop as tm
    ds = L.make_dataset(n_meshes=128, seed0=1000, chunk=128, preset="c5curved", coarse=True)
    assert all(s == tm.OK for s, _, _ in ds.newton)
    net = L.MLP(L.n_features(3), L.n_targets(3), 256, seed=0)
    hist = L.train(net, ds, epochs=12, batch=2048, lr=2e-3)
    print("training loss per epoch:", ["%.3e" % h for h in hist])
    gains = []
    for seed in (5000, 5001):
        m = mg.make_mesh("c5curved", seed)
        ctx = tm.Context.from_mesh(m, precision=tm.FP32_MIXED)
        x0 = torch.tensor(m.x, device="cuda")
        fx = torch.tensor(m.fixed, device="cuda")
        prop = L.propose(net, m, ctx, x0, fx, coarse=True)
        assert prop.used and prop.coarse and prop.F < prop.F0 and prop.min_detA > 0
        g0 = torch.linalg.norm(ctx.gradient(x0)).item()
        xa, xb = x0.clone(), prop.x.clone()
        ra = ctx.newton_solve(xa, max_newton=30, rtol=1e-30, atol=1e-10 * g0)
        rb = ctx.newton_solve(xb, max_newton=30, rtol=1e-30, atol=1e-10 * g0)
        assert ra.status == tm.OK and rb.status == tm.OK
        assert abs(ra.report["F"] - rb.report["F"]) <= 1e-6 * prop.F0
        assert rb.report["min_detA"] > 0
        assert rb.report["krylov_iterations"] < ra.report["krylov_iterations"]
        gains.append((prop.scale, ra.report["krylov_iterations"], rb.report["krylov_iterations"]))
    print("scale kept, krylov without / with the proposal:", gains)
