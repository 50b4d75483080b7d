"""Pins for the oracle's cell-based Delaunay triangulation (Sec. 2.1, 4.1).

The cell-clipping result must equal an independent exact brute-force
Delaunay triangulation (tests/bruteforce.py) filtered by the emission rule
(circumcentre, by the fixed FP64 formula, inside the bounded regions of all
three vertices).  Further pins: hull counts, Euler characteristic, cell areas
summing to the box area, neighbour symmetry.
"""
import math

import numpy as np
import pytest

import bruteforce as bf
import workloads as W

RT = 0.70710678118654752440


def circumcentre_fixed(a, b, c):
    bx, by = b[0] - a[0], b[1] - a[1]
    cx, cy = c[0] - a[0], c[1] - a[1]
    B = bx * bx + by * by
    C = cx * cx + cy * cy
    D = 2.0 * (bx * cy - by * cx)
    ux = (cy * B - by * C) / D
    uy = (bx * C - cx * B) / D
    return a[0] + ux, a[1] + uy


def in_box(c, g):
    return g.x0 <= c[0] <= g.x1 and g.y0 <= c[1] <= g.y1


def in_oct(c, p, S):
    dx, dy = c[0] - p[0], c[1] - p[1]
    return abs(dx) <= S and abs(dy) <= S and abs(RT * (dx + dy)) <= S and abs(RT * (dy - dx)) <= S


def big_disk():
    sdf = W.grid_from_fn(lambda x, y: W.disk_sdf_fn(x, y, r=1.0), 64)
    return sdf, W.constant_grid(1.0)


def test_unbounded_equals_bruteforce(oracle_mod):
    sdf, siz = big_disk()
    rng = np.random.default_rng(3)
    for trial in range(4):
        n = 22
        pts = rng.uniform(-0.9, 0.9, (n, 2))
        m = oracle_mod.OracleMesh(sdf, siz, pts, bounded=0, validity=0)
        m.rebuild()
        got = [tuple(t) for t in m.triangles()]
        dt = bf.delaunay([tuple(p) for p in pts])
        want = [t for t in dt if in_box(circumcentre_fixed(pts[t[0]], pts[t[1]], pts[t[2]]), sdf)]
        assert got == sorted(want), trial


def test_bounded_equals_filtered_bruteforce(oracle_mod):
    sdf, _ = big_disk()
    # strongly varying sizing so octagon bounds cut real Delaunay triangles
    siz = W.grid_from_fn(lambda x, y: 0.02 + 0.3 * (x + 1.1), 16)
    rng = np.random.default_rng(5)
    for trial in range(3):
        n = 30
        pts = rng.uniform(-0.8, 0.8, (n, 2))
        m = oracle_mod.OracleMesh(sdf, siz, pts, validity=0)
        m.rebuild()
        cls, h, geps, havg = m.geometry()
        dx = (sdf.x1 - sdf.x0) / (sdf.nx - 1)
        dy = (sdf.y1 - sdf.y0) / (sdf.ny - 1)

        def S(p):
            gi = min(max(int(math.floor((p[0] - sdf.x0) / dx)), 0), sdf.nx - 2)
            gj = min(max(int(math.floor((p[1] - sdf.y0) / dy)), 0), sdf.ny - 2)
            return 5.0 * h[gj, gi]

        dt = bf.delaunay([tuple(p) for p in pts])
        want = []
        for t in dt:
            c = circumcentre_fixed(pts[t[0]], pts[t[1]], pts[t[2]])
            if in_box(c, sdf) and all(in_oct(c, pts[v], S(pts[v])) for v in t):
                want.append(t)
        got = [tuple(t) for t in m.triangles()]
        assert got == sorted(want), trial
        assert len(want) < len(dt)  # the bound is active in this fixture


def test_square_lattice_sos(oracle_mod):
    sdf, siz = big_disk()
    pts = W.lattice_points("square", 5, 0.0625)
    m = oracle_mod.OracleMesh(sdf, siz, pts, bounded=0, validity=0)
    m.rebuild()
    got = m.triangles()
    want = bf.delaunay([tuple(p) for p in pts])
    assert [tuple(t) for t in got] == want
    # a triangulation of the lattice square: 2 triangles per lattice cell
    assert len(got) == 2 * 4 * 4
    area = sum(abs(bf.orient(pts[a], pts[b], pts[c])) for a, b, c in got) / 2
    assert float(area) == pytest.approx((4 * 0.0625) ** 2, rel=0, abs=1e-15)
    # deterministic across runs
    m2 = oracle_mod.OracleMesh(sdf, siz, pts, bounded=0, validity=0)
    m2.rebuild()
    assert np.array_equal(m2.triangles(), got)


def test_hex_lattice_unique(oracle_mod):
    sdf, siz = big_disk()
    pts = W.lattice_points("hex", 6, 0.1)
    m = oracle_mod.OracleMesh(sdf, siz, pts, bounded=0, validity=0)
    m.rebuild()
    assert [tuple(t) for t in m.triangles()] == bf.delaunay([tuple(p) for p in pts])


def _hull_size(pts):
    from scipy.spatial import ConvexHull

    return len(ConvexHull(pts).vertices)


def test_hull_counts_on_bruteforce(oracle_mod):
    rng = np.random.default_rng(8)
    pts = rng.uniform(-0.5, 0.5, (20, 2))
    dt = bf.delaunay([tuple(p) for p in pts])
    V, H = len(pts), _hull_size(pts)
    edges = {tuple(sorted((t[a], t[(a + 1) % 3]))) for t in dt for a in range(3)}
    assert len(dt) == 2 * V - 2 - H
    assert len(edges) == 3 * V - 3 - H


def _euler(tri):
    v = len(np.unique(tri))
    e = {tuple(sorted((t[a], t[(a + 1) % 3]))) for t in tri for a in range(3)}
    return v - len(e) + len(tri)


def test_euler_disk_and_annulus(oracle_mod):
    wl = W.disk_workload(n=1500)
    m = oracle_mod.OracleMesh(wl.sdf, wl.sizing, wl.points)
    m.rebuild()
    for _ in range(5):
        m.step()
    m.rebuild()
    assert _euler(m.triangles()) == 1
    wa = W.annulus_workload(n=3000, sdf_n=256, siz_n=128)
    ma = oracle_mod.OracleMesh(wa.sdf, wa.sizing, wa.points, method=1)
    for _ in range(8):
        ma.step()
    ma.rebuild()
    assert _euler(ma.triangles()) == 0


def _shoelace(poly):
    x, y = poly[:, 0], poly[:, 1]
    return 0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y)


def test_cell_areas_sum_to_box_and_symmetry(oracle_mod):
    sdf, siz = big_disk()
    rng = np.random.default_rng(9)
    pts = rng.uniform(-1.05, 1.05, (60, 2))
    m = oracle_mod.OracleMesh(sdf, siz, pts, bounded=0, validity=0)
    m.rebuild()
    total = sum(_shoelace(m.cell_polygon(i)) for i in range(len(pts)))
    assert total == pytest.approx((sdf.x1 - sdf.x0) * (sdf.y1 - sdf.y0), rel=1e-13)
    nb = [set(int(v) for v in m.ring(i) if v >= 0) for i in range(len(pts))]
    for i in range(len(pts)):
        for j in nb[i]:
            assert i in nb[j]


def test_duplicate_points_resolved(oracle_mod):
    sdf, siz = big_disk()
    pts = np.array([[0.0, 0.0], [0.1, 0.0], [0.0, 0.1], [0.1, 0.0], [-0.1, -0.05]])
    m = oracle_mod.OracleMesh(sdf, siz, pts, bounded=0, validity=0)
    m.rebuild()
    tri = m.triangles()
    # the duplicate with the smaller id has an empty cell (SoS: larger id owns it)
    assert 1 not in tri
    assert len(m.ring(1)) == 0 and len(m.ring(3)) > 0


def test_sample_triangles_are_the_owned_subset():
    # Procedure I on a subset of cells yields exactly the full rebuild's
    # triangles whose smallest vertex is in the subset
    import oracle
    import workloads as W

    wl = W.disk_workload(n=3000, seed=3)
    om = oracle.OracleMesh(wl.sdf, wl.sizing, wl.points)
    om.rebuild()
    full = om.triangles()
    cells = np.random.default_rng(1).choice(3000, 400, replace=False)
    sub = om.sample_triangles(cells)
    want = full[np.isin(full[:, 0], cells)]
    key = lambda t: sorted(map(tuple, t.tolist()))
    assert len(sub) == len(want) > 0
    assert key(sub) == key(want)
