"""Argument validation of the C ABI happens on the host before any CUDA call,
so these run without a GPU: bad inputs return TRIME_EINVAL with a message."""
import ctypes as C

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def g():
    import paper_2309_13824_gb300 as g

    g.build()
    return g


def _init(g, sdf, siz, pts, **kw):
    p = g.mesh_default_params()
    for k, v in kw.items():
        setattr(p, k, v)
    gs, a = g._grid(sdf)
    gz, b = g._grid(siz)
    h = C.c_void_p()
    xy = np.ascontiguousarray(pts, dtype=np.float64)
    return g.lib().mesh_init(C.byref(h), C.byref(gs), C.byref(gz), xy.ctypes.data_as(C.c_void_p), len(xy),
                             C.byref(p), None)


def test_invalid_arguments(g):
    sdf = W.grid_from_fn(W.disk_sdf_fn, 32)
    siz = W.constant_grid(1.0)
    ok = np.array([[0.0, 0.0], [0.1, 0.0]])
    assert _init(g, sdf, siz, np.array([[np.nan, 0.0]])) == g.TRIME_EINVAL
    assert "not finite" in g.mesh_last_error()
    assert _init(g, sdf, siz, np.array([[5.0, 0.0]])) == g.TRIME_EINVAL
    assert _init(g, sdf, W.constant_grid(-1.0), ok) == g.TRIME_EINVAL
    assert _init(g, sdf, siz, ok, method=7) == g.TRIME_EINVAL
    assert _init(g, sdf, siz, ok, precision=3) == g.TRIME_EINVAL
    bad = W.Grid(np.zeros((1, 5), dtype=np.float32), -1, -1, 1, 1)
    assert _init(g, bad, siz, ok) == g.TRIME_EINVAL
    outside = W.grid_from_fn(lambda x, y: np.ones_like(x), 16)  # no inner cell anywhere
    assert _init(g, outside, siz, ok) == g.TRIME_EINVAL
    assert g.lib().mesh_step(None, 1, None) == g.TRIME_EINVAL
    assert g.lib().mesh_bucket_points(None, None, 10, 0, 0, 1, 1, 0, 4, None, None, None, None) == g.TRIME_EINVAL


def _batch_init(g, meshes, n_meshes=None, **kw):
    p = g.mesh_default_params()
    for k, v in kw.items():
        setattr(p, k, v)
    nm = len(meshes)
    G = (g.mesh_grid2d * max(nm, 1))()
    Z = (g.mesh_grid2d * max(nm, 1))()
    X = (C.c_void_p * max(nm, 1))()
    N = (C.c_int64 * max(nm, 1))()
    keep = []
    for k, (sdf, siz, pts) in enumerate(meshes):
        gs, a = g._grid(sdf)
        gz, b = g._grid(siz)
        xy = np.ascontiguousarray(pts, dtype=np.float64)
        G[k], Z[k], X[k], N[k] = gs, gz, xy.ctypes.data_as(C.c_void_p), len(xy)
        keep += [a, b, xy]
    h = C.c_void_p()
    return g.lib().mesh_batch_init(C.byref(h), nm if n_meshes is None else n_meshes, G, Z, X, N, C.byref(p), 0,
                                   None)


def test_invalid_batch_arguments(g):
    sdf = W.grid_from_fn(W.disk_sdf_fn, 32)
    siz = W.constant_grid(1.0)
    ok = np.array([[0.0, 0.0], [0.1, 0.0]])
    assert _batch_init(g, [], n_meshes=0) == g.TRIME_EINVAL
    assert _batch_init(g, [(sdf, siz, ok), (sdf, siz, np.array([[7.0, 0.0]]))]) == g.TRIME_EINVAL
    assert "mesh 1" in g.mesh_last_error()
    assert _batch_init(g, [(sdf, W.constant_grid(0.0), ok)]) == g.TRIME_EINVAL
    assert "mesh 0" in g.mesh_last_error()
    assert _batch_init(g, [(sdf, siz, ok)], method=9) == g.TRIME_EINVAL
    assert g.lib().mesh_batch_step(None, 1, None) == g.TRIME_EINVAL
    assert g.lib().mesh_batch_get_triangles(None, 0, None, 0, None) == g.TRIME_EINVAL
    assert g.lib().mesh_batch_size(None) == 0


def test_segment_sdf_invalid_arguments(g):
    out = np.zeros((8, 8), np.float32)
    tri = np.array([[0.0, 0.0], [0.0, 1.0], [1.0, 0.0]])

    def call(v, box=(-1, -1, 1, 1), n=8):
        v = np.ascontiguousarray(v, dtype=np.float64)
        return g.lib().mesh_segment_sdf_grid(v.ctypes.data_as(C.POINTER(C.c_double)), len(v), *box, n, n,
                                             out.ctypes.data_as(C.c_void_p), None)

    assert call(tri[:2]) == g.TRIME_EINVAL
    assert call(np.array([[0.0, 0.0], [0.0, 0.0], [1.0, 0.0]])) == g.TRIME_EINVAL
    assert "zero-length" in g.mesh_last_error()
    assert call(np.array([[0.0, np.inf], [0.0, 1.0], [1.0, 0.0]])) == g.TRIME_EINVAL
    assert call(tri, box=(1, -1, -1, 1)) == g.TRIME_EINVAL
    assert call(tri, n=1) == g.TRIME_EINVAL


def test_init_points_invalid_arguments(g):
    sdf = W.grid_from_fn(W.disk_sdf_fn, 32)
    gs, a = g._grid(sdf)
    gz, b = g._grid(W.constant_grid(1.0))
    n = C.c_int64()
    assert g.lib().mesh_init_points(C.byref(gs), C.byref(gz), 0, 1, None, None, 0, C.byref(n), None) == g.TRIME_EINVAL
    gneg, c = g._grid(W.constant_grid(-1.0))
    assert g.lib().mesh_init_points(C.byref(gs), C.byref(gneg), 10, 1, None, None, 0, C.byref(n), None) == g.TRIME_EINVAL


def test_adf_invalid_arguments(g):
    L = g.lib()
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    sq = np.ascontiguousarray([[-0.5, -0.5], [-0.5, 0.5], [0.5, 0.5], [0.5, -0.5]], dtype=np.float64)
    cells = np.array([0, 5, 9], np.int32)
    tol = np.full(3, 1e-4)
    h = C.c_void_p()

    def build(v=sq, nv=4, box=(-1.0, -1.0, 1.0, 1.0), n=9, c=cells, t=tol, depth=10):
        return L.mesh_adf_build(v.ctypes.data_as(dp), nv, *box, n, n, c.ctypes.data_as(ip), t.ctypes.data_as(dp),
                                len(c), depth, C.byref(h), None)

    assert build(nv=2) == g.TRIME_EINVAL
    assert build(box=(1.0, -1.0, -1.0, 1.0)) == g.TRIME_EINVAL
    assert build(depth=15) == g.TRIME_EINVAL and "max_depth" in g.mesh_last_error()
    assert build(c=np.array([0, 5, 5], np.int32)) == g.TRIME_EINVAL and "distinct" in g.mesh_last_error()
    assert build(c=np.array([0, 5, 64], np.int32)) == g.TRIME_EINVAL  # 8 x 8 cells
    assert build(t=np.array([1e-4, -1.0, 1e-4])) == g.TRIME_EINVAL
    bad = sq.copy()
    bad[1, 0] = np.inf
    assert build(v=bad) == g.TRIME_EINVAL and "finite" in g.mesh_last_error()
    assert not h.value  # nothing was built
    pts = np.zeros((4, 2))
    out = np.zeros(4)
    assert L.mesh_segment_sdf_points(sq.ctypes.data_as(dp), 2, pts.ctypes.data_as(C.c_void_p), 4,
                                     out.ctypes.data_as(C.c_void_p), None) == g.TRIME_EINVAL
    assert L.mesh_adf_eval(None, pts.ctypes.data_as(C.c_void_p), 4, out.ctypes.data_as(C.c_void_p),
                           None) == g.TRIME_EINVAL
