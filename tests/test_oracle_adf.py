"""Pins of the oracle's adaptive distance field (Sec. 3.7, Fig. 17; App. B
T_depth = 10, fac_Etol = 0.1): the quadtree structure, the corner values
against the exact segment SDF, the subdivision rule re-evaluated from its
definition, and closed forms (an affine SDF never splits)."""
import numpy as np

import oracle as O


def _square(h=0.5):
    return np.array([[-h, -h], [-h, h], [h, h], [h, -h]])  # clockwise


def _regular(k, r):
    th = -2 * np.pi * np.arange(k) / k
    return r * np.stack([np.cos(th), np.sin(th)], 1)


def _corner_xy(box, nx, ny, cells, root, lev):
    """Node corner coordinates by the fixed formula cx0 + ix (dx 2^-L)."""
    x0, y0, x1, y1 = box
    dx, dy = (x1 - x0) / (nx - 1), (y1 - y0) / (ny - 1)
    c = np.asarray(cells)[root]
    cx0 = x0 + (c % (nx - 1)).astype(float) * dx
    cy0 = y0 + (c // (nx - 1)).astype(float) * dy
    L, ix, iy = lev[:, 0], lev[:, 1], lev[:, 2]
    wx, wy = dx * (1.0 / (1 << L).astype(float)), dy * (1.0 / (1 << L).astype(float))
    xa, xb = cx0 + ix * wx, cx0 + (ix + 1) * wx
    ya, yb = cy0 + iy * wy, cy0 + (iy + 1) * wy
    return xa, xb, ya, yb


def _boundary_cells(v, box, nx, ny):
    """Cells whose corner SDF values change sign or come near zero."""
    x0, y0, x1, y1 = box
    xs, ys = np.linspace(x0, x1, nx), np.linspace(y0, y1, ny)
    X, Y = np.meshgrid(xs, ys)
    s = O.segment_sdf(v, X.ravel(), Y.ravel()).reshape(ny, nx)
    lo = np.minimum(np.minimum(s[:-1, :-1], s[:-1, 1:]), np.minimum(s[1:, :-1], s[1:, 1:]))
    hi = np.maximum(np.maximum(s[:-1, :-1], s[:-1, 1:]), np.maximum(s[1:, :-1], s[1:, 1:]))
    j, i = np.nonzero((lo <= 0.02) & (hi >= -0.02))
    return (j * (nx - 1) + i).astype(np.int32)


def test_structure_and_corner_values():
    v = _regular(7, 0.7)
    box, nx, ny = (-1.0, -1.0, 1.0, 1.0), 33, 33
    cells = _boundary_cells(v, box, nx, ny)
    a = O.OracleADF(v, box, nx, ny, cells, np.full(len(cells), 1e-5), max_depth=6)
    V, child, root, lev = a.nodes()
    n = len(V)
    assert n > len(cells)
    # level 0 is the cell list in order
    assert np.array_equal(root[: len(cells)], np.arange(len(cells))) and np.all(lev[: len(cells)] == 0)
    # children: four consecutive nodes one level down, quadrants (0,0),(1,0),(0,1),(1,1)
    par = np.nonzero(child >= 0)[0]
    for k in par:
        c = child[k] + np.arange(4)
        assert np.all(root[c] == root[k]) and np.all(lev[c, 0] == lev[k, 0] + 1)
        assert np.array_equal(lev[c, 1], 2 * lev[k, 1] + np.array([0, 1, 0, 1]))
        assert np.array_equal(lev[c, 2], 2 * lev[k, 2] + np.array([0, 0, 1, 1]))
    # levels never decrease in build order and every non-root node has a parent
    assert np.all(np.diff(lev[:, 0]) >= 0)
    assert len(par) * 4 == n - len(cells)
    # every corner holds the exact SDF at its coordinates
    xa, xb, ya, yb = _corner_xy(box, nx, ny, cells, root, lev)
    for col, (px, py) in enumerate(((xa, ya), (xb, ya), (xa, yb), (xb, yb))):
        assert np.array_equal(V[:, col], O.segment_sdf(v, px, py))


def test_subdivision_rule_from_its_definition():
    v = _regular(5, 0.6)
    box, nx, ny = (-1.0, -1.0, 1.0, 1.0), 17, 17
    cells = _boundary_cells(v, box, nx, ny)
    tol = np.where(np.arange(len(cells)) % 2 == 0, 1e-4, 3e-6)
    depth = 7
    a = O.OracleADF(v, box, nx, ny, cells, tol, max_depth=depth)
    V, child, root, lev = a.nodes()
    xa, xb, ya, yb = _corner_xy(box, nx, ny, cells, root, lev)
    xm, ym = 0.5 * (xa + xb), 0.5 * (ya + yb)
    s = [O.segment_sdf(v, px, py) for px, py in ((xm, ya), (xm, yb), (xa, ym), (xb, ym), (xm, ym))]
    p = [(V[:, 0] + V[:, 1]) * 0.5, (V[:, 2] + V[:, 3]) * 0.5, (V[:, 0] + V[:, 2]) * 0.5, (V[:, 1] + V[:, 3]) * 0.5,
         ((V[:, 0] + V[:, 1]) + (V[:, 2] + V[:, 3])) * 0.25]
    err = np.max(np.abs(np.array(p) - np.array(s)), axis=0)
    split = (err > tol[root]) & (lev[:, 0] < depth)
    assert np.array_equal(child >= 0, split)
    assert split.any() and (~split).any()


def test_affine_sdf_never_splits_and_is_exact():
    # cells along the middle of the square's edges: the SDF is affine there
    v = _square(0.5)
    box, nx, ny = (-1.0, -1.0, 1.0, 1.0), 41, 41  # dx = 0.05
    dx = 0.05
    cells = []
    for t in (16, 18, 20, 22):  # columns near x = 0, the cells straddling y = 0.5
        cells.append(int(round((0.5 + 1.0) / dx)) * (nx - 1) + t)
    a = O.OracleADF(v, box, nx, ny, np.array(cells), np.zeros(len(cells)), max_depth=5)
    V, child, root, lev = a.nodes()
    # bilinear reproduces an affine function up to rounding, so even a zero
    # tolerance splits only where rounding leaves a residue
    rng = np.random.default_rng(0)
    px = -0.2 + 0.4 * rng.random(2000)
    py = 0.5 + dx * rng.random(2000) - 1e-12
    got = a.eval(px, py)
    ok = ~np.isnan(got)
    assert ok.sum() > 1000
    assert np.abs(got[ok] - (py[ok] - 0.5)).max() < 1e-14
    b = O.OracleADF(v, box, nx, ny, np.array(cells), np.full(len(cells), 1e-12), max_depth=5)
    assert len(b.nodes()[0]) == len(cells)  # roots only


def test_depth_caps_and_full_trees():
    v = _regular(9, 0.55)
    box, nx, ny = (-1.0, -1.0, 1.0, 1.0), 9, 9
    cells = _boundary_cells(v, box, nx, ny)
    a0 = O.OracleADF(v, box, nx, ny, cells, np.zeros(len(cells)), max_depth=0)
    assert len(a0.nodes()[0]) == len(cells)
    # zero tolerance on a curved field: every node splits down to the cap
    curved = np.array([c for c in cells])
    a2 = O.OracleADF(v, box, nx, ny, curved, np.zeros(len(curved)), max_depth=2)
    V, child, root, lev = a2.nodes()
    per = np.bincount(root, minlength=len(curved))
    assert np.all((per == 1) | (per == 5) | (per == 21) | (per % 4 == 1))
    assert per.max() == 21


def test_eval_accuracy_and_corner_exactness():
    v = _regular(6, 0.65)
    box, nx, ny = (-1.0, -1.0, 1.0, 1.0), 21, 21
    cells = _boundary_cells(v, box, nx, ny)
    tol = 2e-6
    a = O.OracleADF(v, box, nx, ny, cells, np.full(len(cells), tol), max_depth=10)
    V, child, root, lev = a.nodes()
    # a leaf's lower-left corner (away from the cell's own edges, which the
    # neighbouring cell may own) leads the descent to that leaf, where the ADF
    # is its corner value: the exact SDF, bit for bit
    xa, xb, ya, yb = _corner_xy(box, nx, ny, cells, root, lev)
    leaf = (child < 0) & (lev[:, 1] > 0) & (lev[:, 2] > 0)
    assert leaf.sum() > 500
    assert np.array_equal(a.eval(xa[leaf], ya[leaf]), V[leaf, 0])
    assert np.array_equal(V[leaf, 0], O.segment_sdf(v, xa[leaf], ya[leaf]))
    # random points of the listed cells: within a few tolerances of the exact SDF
    rng = np.random.default_rng(3)
    dx = 2.0 / (nx - 1)
    c = cells[rng.integers(0, len(cells), 20000)]
    px = -1.0 + (c % (nx - 1) + rng.random(len(c))) * dx
    py = -1.0 + (c // (nx - 1) + rng.random(len(c))) * dx
    err = np.abs(a.eval(px, py) - O.segment_sdf(v, px, py))
    assert err.max() < 8 * tol, err.max()
    # points outside the listed cells have no value
    assert np.isnan(a.eval([0.0], [0.0]))[0]
