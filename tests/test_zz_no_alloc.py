"""tmop_energy_noalloc: the objective and min det A for callers that may not
allocate GPU memory (e.g. an application whose own allocator owns the GPU,
or code inside another program's time step). It keeps its partial sums in
one fixed file-scope device array instead of a context's workspace.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test. It must pass both alone in a
fresh process and after the other tests (the array keeps whatever the last
call left in it)."""
import ctypes as C

import numpy as np
import pytest

from paper_1807_09807_gb300 import meshgen as mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-12   # the FP64 tolerance of the other parity tests


@pytest.fixture(scope="module")
def tm():
    from paper_1807_09807_gb300 import build as cuda_build
    cuda_build.build()
    from paper_1807_09807_gb300 import tmop
    tmop.load()
    return tmop


def _call_capi(tm, m, F, md, metric=None, target_kind=0, scale=1.0):
    """Call the entry point through the C ABI (ctypes, raw device pointers)."""
    lib = tm.load()
    st = (C.c_int * 3)(*(list(m.nx) + [0] * (3 - len(m.nx))))
    q = tm._Quad(m.quad_kind, m.nq)
    t = tm._Targets(target_kind, scale, None)
    x = torch.tensor(m.x, device="cuda")
    rc = lib.tmop_energy_noalloc(m.dim, m.order, st, C.byref(q), metric or m.metric, C.byref(t),
                                 C.c_void_p(x.data_ptr()), C.c_void_p(F.data_ptr()), C.c_void_p(md.data_ptr()),
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, x


@pytest.mark.parametrize("name,kw", [("c3", {}), ("c2", dict(nx=48))])
def test_noalloc_matches_tmop_energy_twice(tm, name, kw):
    m = mg.make_mesh(name, 1, **kw)
    ctx = tm.Context.from_mesh(m)
    F = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
    md = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):                      # two calls in a row share the scratch
        rc, x = _call_capi(tm, m, F, md)
        assert rc == tm.OK
        rc_ref, F_ref, md_ref = ctx.energy(x)
        assert rc_ref == tm.OK
        assert abs(F.item() - F_ref) <= RTOL * abs(F_ref), (call, F.item(), F_ref)
        assert abs(md.item() - md_ref) <= RTOL * abs(md_ref), (call, md.item(), md_ref)


def test_noalloc_smaller_call_after_larger_and_scaled_target(tm):
    big = mg.make_mesh("c3", 2)
    small = mg.make_mesh("c3", 3, nx=3)
    F = torch.empty((), dtype=torch.float64, device="cuda")
    md = torch.empty((), dtype=torch.float64, device="cuda")
    for m in (big, small):
        rc, x = _call_capi(tm, m, F, md, target_kind=tm.W_SCALED, scale=0.5)
        assert rc == tm.OK
        rc_ref, F_ref, md_ref = tm.Context.from_mesh(m, target_scale=0.5).energy(x)
        assert abs(F.item() - F_ref) <= RTOL * abs(F_ref)
        assert abs(md.item() - md_ref) <= RTOL * abs(md_ref)


def test_noalloc_rejects_grids_beyond_its_scratch(tm):
    # 1024 x 1024 order-1 quads need at least 131 072 blocks of partials (at
    # most 8 elements per block) > 32 768: refused on the host before anything
    # is launched
    F = torch.empty((), dtype=torch.float64, device="cuda")
    md = torch.empty((), dtype=torch.float64, device="cuda")
    x = torch.zeros((2, 1025 * 1025), dtype=torch.float64, device="cuda")
    rc = tm.energy_noalloc(2, 1, [1024, 1024], 2, 2, x, F, md)
    assert rc == tm.ERR_CAPACITY
    assert "scratch" in tm.status_string(rc)
    assert tm.energy_noalloc(2, 1, [4, 4], 2, 2, x[:, :25].contiguous(), F, md, target_kind=tm.W_PER_QP) == tm.ERR_ARG


@pytest.mark.parametrize("name,kw", [("c1", {}), ("c3", dict(nx=4))])
def test_noalloc_matches_the_oracle(tm, name, kw):
    """The same entry point against the FP64 CPU oracle of eq. (2.4) (not
    only against the library's own context), on a 2D and a 3D grid."""
    import oracle
    m = mg.make_mesh(name, 1, **kw)
    F = torch.empty((), dtype=torch.float64, device="cuda")
    md = torch.empty((), dtype=torch.float64, device="cuda")
    rc, _ = _call_capi(tm, m, F, md)
    assert rc == tm.OK
    _, Fo, mdo = oracle.Problem(m.dim, m.order, m.elem_nodes, m.nnode, m.fixed, m.nq, m.metric).energy(m.x)
    assert abs(F.item() - Fo) <= RTOL * abs(Fo), (F.item(), Fo)
    assert abs(md.item() - mdo) <= RTOL * abs(mdo), (md.item(), mdo)
