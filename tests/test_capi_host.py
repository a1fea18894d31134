"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every symbol include/tmop.h declares, and rejects
invalid arguments before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1807_09807_gb300 import build as cuda_build
from paper_1807_09807_gb300 import tmop as tm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return tm.load()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?(?:int|void|char\s*\*|const char\*)\s+(tmop_\w+)\s*\(", txt, re.M))
            names |= set(re.findall(r"\b(tmop_\w+)\s*\(", txt))
    return sorted(n for n in names if not n.endswith("_t"))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "tmop_setup" in names and "tmop_hess_apply" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(tm._SIGNATURES) <= set(names)


def test_status_strings(lib):
    assert tm.status_string(0) == "ok"
    assert "inverted" in tm.status_string(3)
    assert "line search" in tm.status_string(4)


def _setup(lib, dim=2, nelem=1, nnode=9, order=2, nq=4, metric=2, precision=0, en=None, structured=(0, 0, 0),
           tkind=0, scale=1.0, W=None, qkind=0):
    en = np.arange(9, dtype=np.int32) if en is None else en
    m = tm._Mesh(dim, nelem, nnode, en.ctypes.data if en is not None else None, None, (C.c_int * 3)(*structured))
    q = tm._Quad(qkind, nq)
    t = tm._Targets(tkind, scale, None if W is None else W.ctypes.data)
    h = C.c_void_p()
    rc = lib.tmop_setup(C.byref(m), order, C.byref(q), metric, C.byref(t), precision, C.byref(h))
    return rc, h


@pytest.mark.parametrize("kw", [
    dict(dim=4), dict(order=0), dict(order=5), dict(nq=1), dict(nq=9), dict(metric=303), dict(metric=5),
    dict(precision=7), dict(qkind=3), dict(nelem=0),
    dict(en=np.array([0, 1, 2, 3, 4, 5, 6, 7, 9], dtype=np.int32)),      # node id out of range
    dict(en=np.array([0, 1, 2, 3, 4, 5, 6, 7, -1], dtype=np.int32)),
    dict(structured=(2, 1, 0)),                                         # inconsistent with nelem/nnode
    dict(tkind=2, scale=-1.0),                                          # det W <= 0
    dict(tkind=1, W=np.array([[1.0, 2.0], [2.0, 1.0]])),                # det W < 0
    dict(tkind=9),
])
def test_setup_rejects_invalid_arguments(lib, kw):
    rc, h = _setup(lib, **kw)
    assert rc == tm.ERR_ARG and not h.value


def test_structured_mismatch_with_table_is_rejected(lib):
    en = np.arange(9, dtype=np.int32)[::-1].copy()       # reversed local order
    rc, h = _setup(lib, en=en, structured=(1, 1, 0))
    assert rc == tm.ERR_ARG


def test_null_arguments(lib):
    assert lib.tmop_energy(None, None, None, None, None) == tm.ERR_ARG
    assert lib.tmop_energy_device(None, None, None, None, None) == tm.ERR_ARG
    assert lib.tmop_gradient(None, None, None, None) == tm.ERR_ARG
    assert lib.tmop_hess_apply(None, None, None, None, None) == tm.ERR_ARG
    assert lib.tmop_gradient_hess_apply(None, None, None, None, None, None) == tm.ERR_ARG
    assert lib.tmop_newton_step(None, None, None, None, None) == tm.ERR_ARG
    assert lib.tmop_newton_solve(None, None, None, None, None) == tm.ERR_ARG
    assert lib.tmop_krylov_solve(None, None, None, None, None, None, None) == tm.ERR_ARG
    assert lib.tmop_linearize(None, None, None) == tm.ERR_ARG
    assert lib.tmop_hess_apply_pa(None, None, None, None) == tm.ERR_ARG
    assert lib.tmop_hess_apply_pa_add(None, None, None, None) == tm.ERR_ARG
    assert lib.tmop_hess_apply_pa_add_f32(None, None, None, None) == tm.ERR_ARG
    assert lib.tmop_energy_gradient(None, None, None, None, None, None) == tm.ERR_ARG
    assert lib.tmop_hessian_diagonal(None, None, None) == tm.ERR_ARG
    assert lib.tmop_element_min_detA(None, None, None, None) == tm.ERR_ARG
    assert lib.tmop_set_composite(None, 0, None, None) == tm.ERR_ARG
    assert lib.tmop_set_restricted_movement(None, 0.0, None, None) == tm.ERR_ARG
    assert lib.tmop_jacobians(None, None, None, None) == tm.ERR_ARG
    assert lib.tmop_set_targets_from_positions(None, 0, None, None) == tm.ERR_ARG
    assert lib.tmop_pa_layout(None, None, None, None) == tm.ERR_ARG
    assert lib.tmop_sizes(None, None, None, None, None) == tm.ERR_ARG
    # empty input: nothing to convert, no device work
    assert lib.tmop_selftest_convert(None, None, None, 0, None) == tm.OK
    assert lib.tmop_selftest_convert(None, None, None, 5, None) == tm.ERR_ARG
    assert lib.tmop_selftest_rcbrt(None, None, 0, None) == tm.OK
    assert lib.tmop_selftest_rcbrt(None, None, 3, None) == tm.ERR_ARG
    assert lib.tmop_vec_axpby(None, 1.0, None, 0.0, 0, None) == tm.OK      # empty: no device work
    assert lib.tmop_vec_axpby(None, 1.0, None, 0.0, 4, None) == tm.ERR_ARG
    assert lib.tmop_vec_add(None, None, 0, None) == tm.OK
    assert lib.tmop_vec_add(None, None, 4, None) == tm.ERR_ARG
    lib.tmop_destroy(None)


def test_compact_product_strides_are_the_search_result():
    """The padded stage-buffer strides compiled into the compact product
    (PacLayout in tmop_pa_compact.cu) are what the bank-conflict search
    returns, for the benchmark's n = 4, q = 5 and the smallest pair."""
    import importlib.util
    csrc = os.path.join(ROOT, "paper_1807_09807_gb300", "csrc")
    spec = importlib.util.spec_from_file_location("pac_layout_search", os.path.join(csrc, "pac_layout_search.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    src = open(os.path.join(csrc, "tmop_pa_compact.cu")).read()
    table = {}
    for line in re.findall(r"^TMOP_PAC_LAYOUT\(([^)]*)\)", src, re.M):
        v = tuple(int(x) for x in line.split(","))
        table[v[:2]] = v[2:]
    assert set(table) == set(mod.PAIRS)
    for pair in ((4, 5), (2, 2)):
        assert table[pair] == mod.search(*pair)
