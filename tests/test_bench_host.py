"""Host-side logic of bench.py's CPU baseline (no GPU): the all-cores oracle
pool rebuilds the caller's mesh in every worker from the seed it was drawn
with, splits the elements into bands of whole z-slabs that cover the mesh
once, and reports a rate from points actually done."""
import numpy as np
import pytest

import bench
from paper_1807_09807_gb300 import meshgen as mg


def test_oracle_pool_bands_cover_whole_slabs():
    m = mg.make_mesh("c3", 1)
    pool = bench.OraclePool(m, procs=3)
    try:
        slab = m.nx[0] * m.nx[1]
        bands = pool.bands
        assert bands[0][0] == 0 and bands[-1][1] == m.nelem
        for (a0, a1), (b0, _) in zip(bands, bands[1:]):
            assert a1 == b0
        assert all(e0 % slab == 0 and e1 % slab == 0 and e1 > e0 for e0, e1 in bands)
        rate, qp, dt = pool.rate(0.5)
        assert qp > 0 and dt >= 0.5 and qp % m.Q == 0
        assert rate == pytest.approx(qp / dt)
    finally:
        pool.close()


def test_oracle_worker_mesh_is_the_callers_mesh():
    # a mesh drawn with a redraw seed is rebuilt from m.seed alone
    m = mg.make_mesh("c1", 1)
    again = mg.make_mesh(m.name, m.seed)
    assert np.array_equal(m.x, again.x) and np.array_equal(m.elem_nodes, again.elem_nodes)
