"""The adaptive distance field (Sec. 3.7) and the exact point SDF on the GPU
against the oracle, through the C ABI: identical trees node for node
(corners, children, roots, levels), identical values at random points, and
the paper's boundary cells and tolerances taken from a mesh."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

BOX = (-1.1, -1.1, 1.1, 1.1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import paper_2309_13824_gb300 as g

    g.build()
    oracle.build()


def _boundary_cells(v, n, band=0.03):
    xs = np.linspace(BOX[0], BOX[2], n)
    X, Y = np.meshgrid(xs, xs)
    s = oracle.segment_sdf(v, X.ravel(), Y.ravel()).reshape(n, n)
    lo = np.minimum(np.minimum(s[:-1, :-1], s[:-1, 1:]), np.minimum(s[1:, :-1], s[1:, 1:]))
    hi = np.maximum(np.maximum(s[:-1, :-1], s[:-1, 1:]), np.maximum(s[1:, :-1], s[1:, 1:]))
    j, i = np.nonzero((lo <= band) & (hi >= -band))
    return (j * (n - 1) + i).astype(np.int32)


def _same_nodes(a, b):
    for x, y in zip(a, b):
        assert x.shape == y.shape
        assert np.array_equal(x, y)


def _points_in(cells, n, k, seed):
    rng = np.random.default_rng(seed)
    d = (BOX[2] - BOX[0]) / (n - 1)
    c = cells[rng.integers(0, len(cells), k)]
    return np.stack([BOX[0] + (c % (n - 1) + rng.random(k)) * d, BOX[1] + (c // (n - 1) + rng.random(k)) * d], 1)


@pytest.mark.parametrize("depth", [0, 3, 10])
def test_adf_matches_oracle(depth):
    import paper_2309_13824_gb300 as g

    v = W.star_polygon(60, 0.45, 1.0, 5)
    n = 129
    cells = _boundary_cells(v, n)
    tol = np.where(np.arange(len(cells)) % 3 == 0, 1e-4, 1e-5)
    a = g.ADF(v, BOX, n, n, cells, tol, max_depth=depth)
    o = oracle.OracleADF(v, BOX, n, n, cells, tol, max_depth=depth)
    _same_nodes(a.nodes(), o.nodes())
    nn, levels = a.size()
    assert nn == len(o.nodes()[0]) and levels <= depth + 1
    if depth == 10:
        assert levels > 4
    p = np.concatenate([_points_in(cells, n, 20000, 1), np.random.default_rng(2).uniform(-1.1, 1.1, (5000, 2))])
    got, want = a.eval(p), o.eval(p[:, 0], p[:, 1])
    assert np.array_equal(got, want, equal_nan=True)
    assert np.isnan(got).any() and (~np.isnan(got)).sum() >= 20000


def test_adf_eval_device_buffers_and_edges():
    import torch

    import paper_2309_13824_gb300 as g

    v = W.star_polygon(40, 0.5, 1.0, 7)
    n = 65
    cells = _boundary_cells(v, n, 0.05)
    a = g.ADF(v, BOX, n, n, cells, np.full(len(cells), 1e-5))
    o = oracle.OracleADF(v, BOX, n, n, cells, np.full(len(cells), 1e-5))
    # node corners and cell edges (midpoint ties go to the upper child)
    V, child, root, lev = o.nodes()
    d = (BOX[2] - BOX[0]) / (n - 1)
    c = cells[root]
    w = d / (1 << lev[:, 0]).astype(float)
    cx0, cy0 = BOX[0] + (c % (n - 1)) * d, BOX[1] + (c // (n - 1)) * d
    p = np.stack([cx0 + lev[:, 1] * w, cy0 + lev[:, 2] * w], 1)
    p = np.concatenate([p, np.stack([cx0 + (lev[:, 1] + 0.5) * w, cy0 + lev[:, 2] * w], 1)])
    want = o.eval(p[:, 0], p[:, 1])
    assert np.array_equal(a.eval(p), want, equal_nan=True)
    pd = torch.from_numpy(p).cuda()
    out = torch.empty(len(p), dtype=torch.float64, device="cuda")
    a.eval(pd, out=out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), want, equal_nan=True)
    a.close()


def test_segment_sdf_points_exact():
    import paper_2309_13824_gb300 as g

    v = W.star_polygon(80, 0.4, 1.0, 9)
    rng = np.random.default_rng(4)
    p = rng.uniform(-1.1, 1.1, (30000, 2))
    p = np.concatenate([p, v, 0.5 * (v + np.roll(v, -1, 0))])  # vertices and segment midpoints too
    assert np.array_equal(g.segment_sdf_points(v, p), oracle.segment_sdf(v, p[:, 0], p[:, 1]))


def test_adf_for_mesh_cells_and_tolerances():
    import paper_2309_13824_gb300 as g

    v = W.star_polygon(40, 0.5, 1.0, 3)
    n = 129
    sdf = W.polygon_sdf_grid(v, n, BOX)
    siz = W.constant_grid(0.02)
    pts = W.density_in_grid(sdf, siz, 4000, seed=1)
    m = g.Mesh(sdf, siz, pts)
    a = g.ADF.for_mesh(m, v, sdf, fac_etol=0.1, max_depth=10)
    om = oracle.OracleMesh(sdf, siz, pts)
    cls, h, geps, havg = om.geometry()
    cells = np.nonzero(cls.ravel() == 1)[0].astype(np.int32)
    tol = 0.1 * geps.ravel()[cells] * np.sqrt(len(pts) / len(pts))
    assert np.array_equal(a.cells, cells)
    assert np.allclose(a.tol, tol, rtol=1e-15, atol=0)
    o = oracle.OracleADF(v, (sdf.x0, sdf.y0, sdf.x1, sdf.y1), n, n, cells, tol, max_depth=10)
    _same_nodes(a.nodes(), o.nodes())
    # the refined field is far closer to the exact SDF than the float grid
    p = _points_in(cells, n, 20000, 6)
    exact = oracle.segment_sdf(v, p[:, 0], p[:, 1])
    e_adf = np.abs(a.eval(p) - exact).max()
    e_grid = np.abs(W._bilinear_np(sdf, p[:, 0], p[:, 1]) - exact).max()
    assert e_adf < 0.1 * e_grid, (e_adf, e_grid)
    m.close()
