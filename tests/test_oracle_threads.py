"""The oracle's OpenMP per-cell loops (used only to time it on all host
cores) give exactly the results of one thread: the same rings, triangles,
edges, statistics, moves, classes and counters, step after step."""
import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("method", [0, 1, 2])
def test_threads_do_not_change_results(oracle_mod, method):
    wl = W.annulus_workload(n=6000, seed=5, sdf_n=256, siz_n=128)
    a = oracle_mod.OracleMesh(wl.sdf, wl.sizing, wl.points, method=method)
    b = oracle_mod.OracleMesh(wl.sdf, wl.sizing, wl.points, method=method)
    b.set_threads(5)
    for it in range(4):
        sa, sb = a.step(), b.step()
        assert sa == sb, it
        assert np.array_equal(a.triangles(), b.triangles())
        assert np.array_equal(a.edges(), b.edges())
        assert np.array_equal(a.points(), b.points())
        assert np.array_equal(a.classes(), b.classes())
        assert np.array_equal(a.dprev(), b.dprev())
        for i in (0, 17, 2999, 5999):
            assert np.array_equal(a.ring(i), b.ring(i))
    if method == 1:
        assert np.array_equal(a.quad_level(), b.quad_level())
        assert np.array_equal(a.centroid(), b.centroid())
