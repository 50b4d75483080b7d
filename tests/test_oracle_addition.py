"""Pins of the oracle's point-addition scheme (Sec. 3.6) and of the quantities
it rescales (Sec. 3.7), checked against the paper's worked example, the
definitions written out independently in numpy, and hand-computed counts."""
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

HERE = os.path.dirname(__file__)


def _annulus(n, seed=3):
    return W.annulus_workload(n=n, seed=seed, sdf_n=128, siz_n=64)


def _run_until_added(m, max_iters=400):
    for _ in range(max_iters):
        s = m.step()
        if s["added"]:
            return s
    raise AssertionError("no addition within %d iterations" % max_iters)


def test_figure_example():
    """The caption's example: N_total = 5000, fac_init = 0.2 gives 1000 initial
    points and a first addition of 0.6 x 1000 = 600 points (CVD meshing)."""
    with open(os.path.join(HERE, "golden", "point_addition_example.json")) as f:
        g = {k: v["value"] for k, v in json.load(f).items() if not k.startswith("_")}
    n_init = int(round(g["fac_init"] * g["N_total"]))
    assert n_init == g["N_init"]
    w = _annulus(n_init)
    m = O.OracleMesh(w.sdf, w.sizing, w.points, method=1, n_total=g["N_total"], fac_add=g["fac_add"])
    s = _run_until_added(m)
    assert s["added"] == g["first_N_add"]
    assert s["n_points"] == g["N_init"] + g["first_N_add"] == m.n


def test_addition_counts_and_phase_rules():
    """N_add = min(floor(0.6 N_current), N_total - N_current): 100 -> 160
    (+60) -> 250 (+min(96, 90) = 90).  While N_current < N_total the hybrid
    neither switches nor terminates; the iteration right after an addition
    measures no quality change, so it cannot switch."""
    w = W.disk_workload(n=100, seed=5, sdf_n=128)
    m = O.OracleMesh(w.sdf, w.sizing, w.points, method=2, n_total=250)
    added, after_last = [], None
    for it in range(600):
        s = m.step()
        if s["added"]:
            added.append((s["added"], s["n_points"]))
            assert s["method_used"] == -1 and not s["terminated"]
            if s["n_points"] == 250:
                after_last = it + 1
        if s["n_points"] < 250 or s["added"]:
            assert not s["switched"] and not s["terminated"]
        if it == after_last:
            assert not s["switched"]
        if s["terminated"]:
            break
    assert added == [(60, 160), (90, 250)]
    assert s["terminated"] and s["switched"] and m.n == 250


def _cells(geom_x0, geom_y0, dx, dy, ncx, ncy, x, y):
    gi = np.clip(np.floor((x - geom_x0) / dx), 0, ncx - 1).astype(int)
    gj = np.clip(np.floor((y - geom_y0) / dy), 0, ncy - 1).astype(int)
    return gj * ncx + gi


def _setup_about_to_add(method=2, n=401, n_total=2000, seed=7):
    """A mesh whose next iteration adds points (T_add above any change)."""
    w = _annulus(n, seed=seed)
    m = O.OracleMesh(w.sdf, w.sizing, w.points, method=method, n_total=n_total, T_add=1e9)
    s = m.step()  # no previous quality yet: no addition, a move
    assert s["added"] == 0
    return w, m


def test_selection_against_brute_force():
    """The new points are the centroids of the N_add valid triangles with the
    largest circumradius / h_i (h_i of the centroid's geometry cell), computed
    here with the textbook circumradius abc / (4 area); their indices follow
    the ascending vertex triples of their triangles."""
    w, m = _setup_about_to_add()
    p0 = m.points()
    n0 = len(p0)
    cls_g, h, geps, havg = m.geometry()
    s = m.step()
    nadd = s["added"]
    assert nadd == int(np.floor(0.6 * n0)) == 240  # floor(240.6)
    tri = m.triangles()  # the triangulation the addition read (old indices)
    assert tri.max() < n0
    a, b, c = p0[tri[:, 0]], p0[tri[:, 1]], p0[tri[:, 2]]
    la = np.linalg.norm(b - c, axis=1)
    lb = np.linalg.norm(c - a, axis=1)
    lc = np.linalg.norm(a - b, axis=1)
    area = 0.5 * np.abs((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]))
    R = la * lb * lc / (4 * area)
    g = (a + b + c) / 3.0
    sdf = w.sdf
    dx = (sdf.x1 - sdf.x0) / (sdf.nx - 1)
    dy = (sdf.y1 - sdf.y0) / (sdf.ny - 1)
    ncx, ncy = sdf.nx - 1, sdf.ny - 1
    hc = h.reshape(-1)[_cells(sdf.x0, sdf.y0, dx, dy, ncx, ncy, g[:, 0], g[:, 1])]
    ratio = R / hc
    order = np.argsort(-ratio, kind="stable")
    thr = ratio[order[nadd - 1]]
    # clear-cut triangles (not within rounding of the threshold) decide
    must = np.where(ratio > thr * (1 + 1e-9))[0]
    never = np.where(ratio < thr * (1 - 1e-9))[0]
    new = m.points()[n0:]
    assert len(new) == nadd
    # match every new point to its triangle by centroid
    from scipy.spatial import cKDTree

    d, k = cKDTree(g).query(new)
    assert np.all(d <= 1e-14)
    chosen = set(k.tolist())
    assert len(chosen) == nadd
    assert set(must.tolist()) <= chosen
    assert not (set(never.tolist()) & chosen)
    trip = np.sort(tri[k], axis=1)
    keys = [tuple(t) for t in trip]
    assert keys == sorted(keys)  # indices in ascending triple order


def test_rescaled_quantities_match_definition():
    """After an addition h_i, geps_i and h_avg equal their Sec. 3.7
    definitions for the new N_current (a fresh mesh with that many points),
    i.e. the scale factor is sqrt(N_old / N_current)."""
    w, m = _setup_about_to_add()
    s = m.step()
    n1 = s["n_points"]
    _, h1, geps1, havg1 = m.geometry()
    fresh = O.OracleMesh(w.sdf, w.sizing, _annulus(n1, seed=11).points, method=2)
    _, hf, gepsf, havgf = fresh.geometry()
    assert np.allclose(h1, hf, rtol=1e-14, atol=0)
    assert np.allclose(geps1, gepsf, rtol=1e-14, atol=0)
    assert havg1 == pytest.approx(havgf, rel=1e-14)


def test_new_point_state():
    """New points are classified like initial points (Sec. 3.5 / 4.3 rule,
    outside counting as boundary) with the rescaled geps_i, and start with a
    previous move of h_i."""
    w, m = _setup_about_to_add()
    n0 = m.n
    m.step()
    cls_g, h, geps, _ = m.geometry()
    new = m.points()[n0:]
    sdf = w.sdf
    dx = (sdf.x1 - sdf.x0) / (sdf.nx - 1)
    dy = (sdf.y1 - sdf.y0) / (sdf.ny - 1)
    c = _cells(sdf.x0, sdf.y0, dx, dy, sdf.nx - 1, sdf.ny - 1, new[:, 0], new[:, 1])
    s = W._bilinear_np(sdf, new[:, 0], new[:, 1])
    ge = geps.reshape(-1)[c]
    kind = cls_g.reshape(-1)[c]
    expect = np.where(kind == 0, 0, np.where((kind == 1) & (s < -ge), 0, 1))
    clear = np.abs(np.abs(s) - ge) > 1e-12 * np.maximum(ge, 1e-300)
    got = m.classes()[n0:]
    assert np.array_equal(got[clear], expect[clear])
    assert np.array_equal(m.dprev()[n0:], h.reshape(-1)[c])


def test_distmesh_retriangulates_after_addition():
    """Algorithm 1 with additions: the iteration after an addition always
    re-triangulates (the old triangulation does not cover the new points)."""
    w = _annulus(300, seed=9)
    m = O.OracleMesh(w.sdf, w.sizing, w.points, method=0, n_total=600)
    for _ in range(400):
        s = m.step()
        if s["added"]:
            nxt = m.step()
            assert nxt["triangulated"] == 1
            assert m.triangles().max() == m.n - 1 or m.triangles().max() < m.n
            return
    raise AssertionError("no addition")


def test_no_addition_without_n_total():
    w = _annulus(200, seed=2)
    m = O.OracleMesh(w.sdf, w.sizing, w.points, method=2, T_add=1e9)
    for _ in range(5):
        s = m.step()
        assert s["added"] == 0 and s["n_points"] == 200


def test_no_change_measured_across_an_addition():
    """The quality change is not measured across an addition: with T_add above
    any change, additions come every second iteration, never back to back."""
    w, m = _setup_about_to_add(n_total=5000)
    got = [m.step()["added"] > 0 for _ in range(5)]
    assert got == [True, False, True, False, True]
