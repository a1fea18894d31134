"""torch.autograd.Function around the TMOP energy: forward F (eq. (2.4)),
backward by the adjoint gradient kernel, double backward by the Hessian
action; checked against central finite differences (h = 1e-6), torch's
gradcheck and the FP64 CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_1807_09807_gb300 import meshgen as mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tm():
    from paper_1807_09807_gb300 import build as cuda_build
    cuda_build.build()
    from paper_1807_09807_gb300 import tmop
    tmop.load()
    return tmop


def _orc(m, fixed=True):
    return oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed if fixed else None, m.nq, m.metric)


def test_energy_function_matches_oracle_and_fd(tm):
    """3D order-2 hexes, mu303 (and mu302): adjoint gradient vs central FD
    with h = 1e-6 at every free dof, and vs the oracle gradient."""
    from paper_1807_09807_gb300.autograd import tmop_energy
    for metric in (303, 302):
        m = mg.make_mesh("c3", 1, nx=3, metric=metric)
        ctx = tm.Context.from_mesh(m)
        x = torch.tensor(m.x, device="cuda", requires_grad=True)
        F = tmop_energy(x, ctx)
        F.backward()
        orc = _orc(m)
        _, Fo, _ = orc.energy(m.x)
        assert abs(F.item() - Fo) <= 1e-12 * Fo
        g = x.grad.cpu().numpy()
        go = orc.gradient(m.x)
        assert np.linalg.norm(g - go) <= 1e-12 * np.linalg.norm(go)
        h = 1e-6
        xd = x.detach().clone()
        free = np.argwhere(m.fixed == 0)
        fd = np.zeros(len(free))
        for k, (a, i) in enumerate(free):
            xd[a, i] += h
            fp = ctx.energy(xd)[1]
            xd[a, i] -= 2 * h
            fm = ctx.energy(xd)[1]
            xd[a, i] += h
            fd[k] = (fp - fm) / (2 * h)
        ga = g[free[:, 0], free[:, 1]]
        assert np.abs(fd - ga).max() <= 1e-6 * np.abs(ga).max()


def test_gradcheck_and_double_backward(tm):
    from paper_1807_09807_gb300.autograd import tmop_energy
    m = mg.make_mesh("c3", 2, nx=2, order=1, nq=2)
    m.fixed = np.zeros_like(m.fixed)          # every dof free: FD sees them all
    ctx = tm.Context.from_mesh(m)
    x = torch.tensor(m.x, device="cuda", requires_grad=True)
    # FP64 atomics scatter nodal contributions in a run-dependent order, so two
    # backward passes agree to rounding, not bitwise
    assert torch.autograd.gradcheck(lambda t: tmop_energy(t, ctx), (x,), eps=1e-6, atol=1e-6, rtol=1e-5,
                                    nondet_tol=1e-12)
    # Hessian-vector product through torch == the Hessian-action kernel == oracle
    v = torch.randn_like(x)
    F = tmop_energy(x, ctx)
    (g,) = torch.autograd.grad(F, x, create_graph=True)
    (Hv,) = torch.autograd.grad(g, x, grad_outputs=v)
    yo = _orc(m, fixed=False).hess_apply(m.x, v.cpu().numpy())
    assert np.linalg.norm(Hv.cpu().numpy() - yo) <= 1e-12 * np.linalg.norm(yo)
    assert torch.autograd.gradgradcheck(lambda t: tmop_energy(t, ctx), (x,), eps=1e-6, atol=1e-5, rtol=1e-4,
                                        nondet_tol=1e-12)
