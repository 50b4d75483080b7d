"""Pins for three decision rules of the oracle that the closed-form and
brute-force pins elsewhere do not reach:

* the validity Tests 1-3 of Sec. 4.1 (centroid, edge midpoints, circumcentre),
* the movement clamp T_pt = fac_pt h_i of Sec. 4.3 / 3.7 (h_i of the old
  point's cell),
* the hybrid switch of Sec. 4.2 (relative change of the 1/2-mean of alpha
  below T_switch, App. B).

Every expected outcome below follows from hand geometry on inputs where the
bilinear SDF is exact: the grid spans [0, 8]^2 with unit cells and holds
sdf(x, y) = x - 4.25 (every node value is exact in float32 and a bilinear
interpolant of an affine function is that function), so inner cells are the
columns x in [0, 3), boundary cells [3, 6) and outer cells [6, 8] (midpoint
value against the cell diagonal sqrt(2), Sec. 3.2).  With uniform sizing the
Sec. 3.7 quantities are closed forms: h_i = sqrt(A_sel / N) over the 40
selected cells (inner, and boundary cells whose midpoint value is <= 0.5),
geps_i = 0.01 h_i.  Each case lists the branch it exercises and the planted
mistake it catches.
"""
import math

import numpy as np
import pytest

import workloads as W

SIDE = 8
X_IF = 4.25  # the interface sdf = 0


def _half_plane_grids():
    xs = np.arange(SIDE + 1, dtype=np.float64)
    v = np.tile((xs - X_IF).astype(np.float32), (SIDE + 1, 1))
    sdf = W.Grid(v, 0.0, 0.0, float(SIDE), float(SIDE))
    siz = W.Grid(np.ones((2, 2), dtype=np.float32), 0.0, 0.0, float(SIDE), float(SIDE))
    return sdf, siz


def _circumcentre(a, b, c):
    """Textbook circumcentre: solve 2 (b-a).o = |b|^2-|a|^2, 2 (c-a).o = |c|^2-|a|^2."""
    A = 2.0 * np.array([b - a, c - a])
    r = np.array([b @ b - a @ a, c @ c - a @ a])
    o = np.linalg.solve(A, r)
    return o, float(np.linalg.norm(o - a))


def _column_class(x):
    c = math.floor(x)
    return "inner" if c <= 2 else ("boundary" if c <= 5 else "outer")


# (name, vertices in 1/64 units, expected branch facts, expected validity)
#   facts: centroid class, centroid sdf vs geps, midpoints counted by Test 2,
#   |sdf(c)|/R of Test 3 and the sign of sdf(c)
CASES = [
    # Test 1: centroid in an inner cell -> valid, although Test 3 would
    # discard it (|sdf(c)|/R = 0.84).  Catches: inner cells not accepted.
    ("inner_centroid", [[292, 446], [262, 329], [15, 463]], dict(cls="inner"), True),
    # Test 1: centroid in an outer cell -> invalid, although no midpoint is
    # inside and Test 3 would keep it (0.16).  Catches: outer centroids sent
    # on to Tests 2-3.
    ("outer_centroid", [[430, 495], [492, 257], [414, 164]], dict(cls="outer", count=0, ratio_lt=0.4), False),
    # Test 1: centroid in a boundary cell with sdf = 0.30 > geps -> invalid,
    # although two midpoints are inside and Test 3 would keep it (0.12).
    # Catches: the sdf > geps branch of Test 1 skipped.
    ("boundary_centroid_outside", [[443, 353], [332, 417], [98, 225]],
     dict(cls="boundary", gsdf_gt_geps=True, count=2, ratio_lt=0.4), False),
    # Test 2: three midpoints inside -> valid (Test 3 would discard: 0.72).
    ("three_midpoints", [[123, 94], [286, 355], [198, 98]],
     dict(cls="boundary", gsdf_gt_geps=False, count=3, ratio_gt=0.4), True),
    # Test 2: exactly two midpoints inside -> valid (Test 3 would discard:
    # 0.78).  Catches: a threshold of three midpoints.
    ("two_midpoints", [[114, 99], [311, 254], [250, 482]],
     dict(cls="boundary", gsdf_gt_geps=False, count=2, ratio_gt=0.4), True),
    # Test 2: one midpoint -> Test 3, which discards (0.62).  Catches: a
    # threshold of one midpoint.
    ("one_midpoint_test3_discards", [[330, 371], [222, 149], [261, 92]],
     dict(cls="boundary", gsdf_gt_geps=False, count=1, ratio_gt=0.4), False),
    # Test 2: one midpoint -> Test 3, which keeps it (0.026).  Catches: one
    # midpoint discarded without Test 3 (the other reading of Sec. 4.1).
    ("one_midpoint_test3_keeps", [[237, 194], [120, 266], [437, 307]],
     dict(cls="boundary", gsdf_gt_geps=False, count=1, ratio_lt=0.4), True),
    # Test 3 with sdf(c) < 0: |sdf(c)|/R = 0.418 > 0.4 -> invalid.  Catches:
    # the signed sdf(c) instead of its absolute value.
    ("test3_negative_above", [[494, 65], [205, 434], [97, 445]],
     dict(cls="boundary", gsdf_gt_geps=False, count=1, ratio_gt=0.4, ratio_lt=0.42, osign=-1), False),
    # Test 3 with sdf(c) < 0: 0.392 <= 0.4 -> valid.
    ("test3_negative_below", [[377, 251], [187, 121], [222, 494]],
     dict(cls="boundary", gsdf_gt_geps=False, count=1, ratio_gt=0.38, ratio_lt=0.4, osign=-1), True),
    # Test 3 with sdf(c) > 0: 0.407 > 0.4 -> invalid.
    ("test3_positive_above", [[484, 69], [201, 480], [123, 316]],
     dict(cls="boundary", gsdf_gt_geps=False, count=1, ratio_gt=0.4, ratio_lt=0.42, osign=1), False),
    # Test 3 with sdf(c) > 0: 0.391 <= 0.4 -> valid.  Catches: a threshold
    # other than T_circ = 0.4.
    ("test3_positive_below", [[139, 140], [135, 251], [482, 404]],
     dict(cls="boundary", gsdf_gt_geps=False, count=1, ratio_gt=0.38, ratio_lt=0.4, osign=1), True),
]


def _geps_closed_form(n):
    return 0.01 * math.sqrt(40.0 / n)


def test_half_plane_geometry_closed_form(oracle_mod):
    sdf, siz = _half_plane_grids()
    om = oracle_mod.OracleMesh(sdf, siz, np.array([[1.0, 1.0], [2.0, 1.0], [1.0, 2.0]]))
    cls, h, geps, havg = om.geometry()
    cols = np.array([_column_class(i + 0.5) for i in range(SIDE)])
    want = np.where(cols == "inner", 0, np.where(cols == "boundary", 1, 2))
    # class codes of the oracle's geometry grid: inner 0, boundary 1, outer 2
    assert np.array_equal(cls, np.tile(want, (SIDE, 1)))
    assert np.allclose(h, math.sqrt(40.0 / 3.0), rtol=1e-14, atol=0)
    assert np.allclose(geps, _geps_closed_form(3), rtol=1e-14, atol=0)


@pytest.mark.parametrize("name,verts,facts,valid", CASES, ids=[c[0] for c in CASES])
def test_validity_tests_1_to_3(oracle_mod, name, verts, facts, valid):
    P = np.array(verts, dtype=np.float64) / 64.0
    a, b, c = P
    geps = _geps_closed_form(3)
    # the branch facts, from the analytic SDF and textbook geometry
    g = (a + b + c) / 3.0
    assert _column_class(g[0]) == facts["cls"]
    if "gsdf_gt_geps" in facts:
        assert (g[0] - X_IF > geps) == facts["gsdf_gt_geps"]
    mids = [(a + b) / 2, (b + c) / 2, (c + a) / 2]
    count = sum(_column_class(m[0]) == "inner" or (_column_class(m[0]) == "boundary" and m[0] - X_IF <= geps)
                for m in mids)
    if "count" in facts:
        assert count == facts["count"]
    o, R = _circumcentre(a, b, c)
    ratio = abs(o[0] - X_IF) / R
    if "ratio_lt" in facts:
        assert ratio < facts["ratio_lt"]
    if "ratio_gt" in facts:
        assert ratio > facts["ratio_gt"]
    if "osign" in facts:
        assert np.sign(o[0] - X_IF) == facts["osign"]
    assert 0 < o[0] < SIDE and 0 < o[1] < SIDE  # the circumcentre lies in the domain box
    sdf, siz = _half_plane_grids()
    # three points: the Delaunay triangulation is this one triangle; without
    # the validity tests it is emitted, with them only if valid
    om0 = oracle_mod.OracleMesh(sdf, siz, P, validity=0)
    om0.rebuild()
    assert len(om0.triangles()) == 1
    om = oracle_mod.OracleMesh(sdf, siz, P)
    om.rebuild()
    assert len(om.triangles()) == (1 if valid else 0), name


def test_outer_cell_decides_before_its_values(oracle_mod):
    """Test 1 takes the cell's class first: a centroid in an outer cell is
    invalid even where the interpolated sdf there is negative.  The grid
    above with node (6, 3) set to -1: cell (6, 2) keeps a midpoint value of
    1.5625 > sqrt(2) (outer) while the bilinear value at this triangle's
    centroid is -0.08, and two midpoints lie in boundary cells with
    sdf <= geps, so Test 2 alone would keep it.  (On a 1-Lipschitz field an
    outer cell cannot hold sdf <= geps, so only such a grid tells the rule
    apart from Test 1's sdf > geps branch.)  Catches: outer centroids sent
    on to the sdf test and Tests 2-3."""
    sdf, siz = _half_plane_grids()
    sdf.values[3, 6] = -1.0
    P = np.array([[455, 165], [417, 121], [297, 245]], dtype=np.float64) / 64.0
    g = P.mean(0)
    i, j = int(g[0]), int(g[1])
    c = sdf.values[j:j + 2, i:i + 2].astype(np.float64)
    assert (i, j) == (6, 2) and 0.25 * c.sum() > math.sqrt(2)  # a cell with the spike at a corner
    assert W._bilinear_np(sdf, g[:1], g[1:])[0] < 0
    om0 = oracle_mod.OracleMesh(sdf, siz, P, validity=0)
    om0.rebuild()
    assert len(om0.triangles()) == 1
    _, _, geps, _ = om0.geometry()
    assert np.allclose(geps, _geps_closed_form(3), rtol=1e-14, atol=0)  # the spike selects no new cell
    om = oracle_mod.OracleMesh(sdf, siz, P)
    om.rebuild()
    assert len(om.triangles()) == 0


# ---------------------------------------------------------------- the clamp
def _two_size_grids():
    """sdf = x - 4.25 as above; sizing mu = 1 on the nodes x <= 3 and 2 on
    x >= 4, so the cell midpoints carry mu = 1 (columns 0-2), 1.5 (column 3),
    2 (columns 4-7)."""
    sdf, _ = _half_plane_grids()
    xs = np.arange(SIDE + 1)
    mu = np.where(xs <= 3, 1.0, 2.0).astype(np.float32)
    siz = W.Grid(np.tile(mu, (SIDE + 1, 1)), 0.0, 0.0, float(SIDE), float(SIDE))
    return sdf, siz


def _h_closed_form(mu_cell, n):
    # Sec. 3.7: n^E = rho_norm N, rho = 1/mu^2 normalised over the selected
    # cells (inner columns 0-2 with mu = 1, boundary column 3 (midpoint value
    # -0.75, mu 1.5) and column 4 (0.25, mu 2); column 5 (1.25) is not
    # selected), h = sqrt(cell area / n^E)
    sum_rho = 24 * 1.0 + 8 / 1.5 ** 2 + 8 / 2.0 ** 2
    return math.sqrt(sum_rho / ((1.0 / mu_cell ** 2) * n))


def _clamp_mesh(oracle_mod, n=200):
    sdf, siz = _two_size_grids()
    rng = np.random.default_rng(3)
    pts = np.stack([rng.uniform(0.2, 2.8, n), rng.uniform(0.2, 7.8, n)], 1)
    return oracle_mod.OracleMesh(sdf, siz, pts)


def test_geometry_h_two_sizes(oracle_mod):
    om = _clamp_mesh(oracle_mod)
    _, h, _, _ = om.geometry()
    for col, mu in ((0, 1.0), (2, 1.0), (3, 1.5), (4, 2.0), (7, 2.0)):
        assert h[4, col] == pytest.approx(_h_closed_form(mu, 200), rel=1e-13)


@pytest.mark.parametrize("frac", [0.5, 0.9, 3.0])
def test_clamp_lands_at_fac_pt_h_of_old_cell(oracle_mod, frac):
    """A proposed move longer than T_pt = 0.4 h_i is shortened to exactly
    0.4 h_i along its direction, with h_i of the old point's cell (column 2,
    mu = 1) although the new point lies in column 3 (mu = 1.5, where
    0.4 h would be 0.6 h_old).  Catches: a clamp at 2 T_pt, at h of the new
    cell, or none."""
    om = _clamp_mesh(oracle_mod)
    h_old = _h_closed_form(1.0, 200)
    p_old = np.array([2.95, 4.0625])
    u = np.array([0.8, 0.6])
    p_new = p_old + frac * h_old * u
    pf, cls = om.project(p_old, 0, p_new)
    want = p_old + 0.4 * h_old * u
    assert _column_class(want[0]) == "boundary" and want[0] - X_IF < -0.5  # classifies inner, not projected
    assert cls == 0
    assert np.allclose(pf, want, rtol=0, atol=1e-15)
    assert math.hypot(*(pf - p_old)) == pytest.approx(0.4 * h_old, rel=1e-14)


@pytest.mark.parametrize("frac", [0.1, 0.39])
def test_short_move_not_clamped(oracle_mod, frac):
    om = _clamp_mesh(oracle_mod)
    h_old = _h_closed_form(1.0, 200)
    p_old = np.array([2.95, 4.0625])
    p_new = p_old + frac * h_old * np.array([0.8, 0.6])
    pf, cls = om.project(p_old, 0, p_new)
    assert cls == 0
    assert np.array_equal(pf, p_new)


# ------------------------------------------------------------ hybrid switch
def _hybrid_mesh(oracle_mod):
    wl = W.disk_workload(n=1500, seed=4, sdf_n=96)
    om = oracle_mod.OracleMesh(wl.sdf, wl.sizing, wl.points, method=2)
    qa = om.rebuild()["half_mean_alpha"]
    return om, qa


@pytest.mark.parametrize("rel_change,expect_switch", [
    # previous 1/2-mean above the current one by a relative 0.0014: switch,
    # although the absolute change (0.0014 x prev > 0.0015 for prev > 1.07)
    # would not.  Catches: the absolute change instead of the relative one.
    (0.0014, True),
    # relative change 0.0016 > T_switch: no switch
    (0.0016, False),
    # relative change just below T_switch measured against the previous
    # value (0.999 T_switch), which is just above it against the current
    # value (x prev/cur = 1.0015).  Catches: dividing by the current value.
    (0.0015 * 0.999, True),
])
def test_hybrid_switch_relative_change(oracle_mod, rel_change, expect_switch):
    om, qa = _hybrid_mesh(oracle_mod)
    assert qa > 1.1  # the absolute and relative tests disagree at this size of M_1/2
    prev = qa / (1.0 - rel_change)  # (prev - qa) / prev = rel_change
    assert abs(qa - prev) > 0.0015 or not expect_switch or rel_change < 0.00149
    om.set_method_state(0, prev_a=prev, prev_b=1.0, prev_amax=1.0)
    s = om.step()
    assert s["half_mean_alpha"] == qa  # same positions, same triangulation
    assert bool(s["switched"]) == expect_switch
    assert s["method_used"] == (1 if expect_switch else 0)
    assert not s["terminated"]  # the quality termination waits for the iteration after the switch


def test_hybrid_switch_needs_a_previous_iteration(oracle_mod):
    """The first iteration has no previous 1/2-mean: DistMesh, no switch."""
    om, qa = _hybrid_mesh(oracle_mod)
    s = om.step()
    assert not s["switched"] and s["method_used"] == 0
