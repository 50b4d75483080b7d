"""Pins for the oracle's moves: CVD centroid quadrature (Sec. 2.3, 4.2),
DistMesh forces (Sec. 2.2), point treatment (Sec. 4.3), quality (Sec. 3.6),
and the geometry-grid quantities (Sec. 3.2, 3.7).

Reference values are closed forms, invariants and independent numerical
integration; none come from the code under test.
"""
import math

import numpy as np
import pytest

import workloads as W


def _shoelace_centroid(P):
    x, y = P[:, 0], P[:, 1]
    cr = x * np.roll(y, -1) - np.roll(x, -1) * y
    A = 0.5 * cr.sum()
    cx = ((x + np.roll(x, -1)) * cr).sum() / (6 * A)
    cy = ((y + np.roll(y, -1)) * cr).sum() / (6 * A)
    return np.array([cx, cy]), A


def _convex_polygon(rng, k, r=0.2):
    th = np.sort(rng.uniform(0, 2 * np.pi, k))
    rad = r * rng.uniform(0.6, 1.0, k)
    return np.stack([rad * np.cos(th), rad * np.sin(th)], 1)


def test_uniform_density_centroid_is_shoelace(oracle_mod):
    rng = np.random.default_rng(21)
    siz = W.constant_grid(0.37)
    for _ in range(20):
        P = _convex_polygon(rng, rng.integers(3, 12))
        c, lv = oracle_mod.polygon_centroid(siz, (0.0, 0.0), P, eps_c=1e9)
        want, _ = _shoelace_centroid(P)
        assert lv == 1
        assert np.allclose(c, want, rtol=0, atol=1e-15)


def _dense_weighted_centroid(P, mu_fn, n=700):
    """Independent reference: midpoint rule on a fine fan of sub-triangles."""
    from itertools import product

    W_ = WX = WY = 0.0
    for t in range(len(P)):
        a, b = np.zeros(2), P[t]
        c = P[(t + 1) % len(P)]
        u, v = np.meshgrid((np.arange(n) + 1 / 3) / n, (np.arange(n) + 1 / 3) / n)
        m = u + v < 1
        pts = a + u[m][:, None] * (b - a) + v[m][:, None] * (c - a)
        u2, v2 = np.meshgrid((np.arange(n) + 2 / 3) / n, (np.arange(n) + 2 / 3) / n)
        m2 = u2 + v2 < 1
        pts = np.concatenate([pts, a + u2[m2][:, None] * (b - a) + v2[m2][:, None] * (c - a)])
        area = 0.5 * abs((b - a)[0] * (c - a)[1] - (b - a)[1] * (c - a)[0])
        w = (area / (n * n)) / mu_fn(pts[:, 0], pts[:, 1]) ** 2
        W_ += w.sum(); WX += (w * pts[:, 0]).sum(); WY += (w * pts[:, 1]).sum()
    return np.array([WX / W_, WY / W_])


def test_adaptive_quadrature_converges(oracle_mod):
    # mu linear in x (a 2x2 bilinear grid): rho = 1/mu^2 is not linear, so
    # deeper levels must approach the true weighted centroid
    siz = W.Grid(np.array([[0.05, 1.0], [0.05, 1.0]], dtype=np.float32), -1.1, -1.1, 1.1, 1.1)
    mu = lambda x, y: 0.05 + (x + 1.1) / 2.2 * 0.95
    P = np.array([[-0.9, -0.3], [0.4, -0.35], [0.5, 0.3], [-0.8, 0.45]])
    ref = _dense_weighted_centroid(P, mu)
    errs = []
    for lv in range(1, 8):
        c, got = oracle_mod.polygon_centroid(siz, (0.0, 0.0), P, eps_c=0.0, max_level=lv)
        assert got == lv
        errs.append(np.linalg.norm(c - ref))
    # one-point rule: error O(diameter^2), i.e. about 4x smaller per level pair
    assert errs[-1] < errs[0] / 30
    assert all(errs[k + 2] < errs[k] / 2.5 for k in range(len(errs) - 2))


def test_lloyd_fixed_point_on_hex_lattice(oracle_mod):
    sdf = W.grid_from_fn(lambda x, y: W.disk_sdf_fn(x, y, r=1.0), 64)
    siz = W.constant_grid(1.0)
    pts = W.lattice_points("hex", 12, 0.05)
    m = oracle_mod.OracleMesh(sdf, siz, pts, method=1, bounded=0, validity=0)
    m.set_dprev(np.full(len(pts), 1e-9))
    m.step()
    c = m.centroid()
    # interior generators (two rings away from the lattice hull) are centroids
    r = np.hypot(*(pts - pts.mean(0)).T)
    inner = r < 0.18
    assert inner.sum() > 20
    assert np.abs(c[inner] - pts[inner]).max() < 1e-14


def test_cvd_energy_decreases(oracle_mod):
    sdf = W.grid_from_fn(lambda x, y: W.disk_sdf_fn(x, y, r=5.0), 32)
    siz = W.constant_grid(1.0)
    rng = np.random.default_rng(4)
    pts = rng.uniform(-1.05, 1.05, (40, 2))

    def energy(p):
        m = oracle_mod.OracleMesh(sdf, siz, p, method=1, bounded=0, validity=0)
        m.rebuild()
        E = 0.0
        for i in range(len(p)):
            P = m.cell_polygon(i) - p[i]
            for t in range(len(P)):
                b, c = P[t], P[(t + 1) % len(P)]
                A = 0.5 * (b[0] * c[1] - b[1] * c[0])
                # exact second moment of triangle (0,b,c) about the origin
                E += A / 6 * (b @ b + c @ c + b @ c)
        return E, m

    E0, m = energy(pts)
    m.set_dprev(np.full(len(pts), 1e-9))
    m.step()
    E1, _ = energy(m.points())
    assert E1 < E0


def _dm_mesh(oracle_mod, pts, **kw):
    sdf = W.grid_from_fn(lambda x, y: W.disk_sdf_fn(x, y, r=1.0), 128)
    siz = W.constant_grid(1.0)
    return oracle_mod.OracleMesh(sdf, siz, pts, method=0, **kw)


def test_equilateral_force_closed_form(oracle_mod):
    l = 0.05
    pts = np.array([[0.0, 0.0], [l, 0.0], [l / 2, l * math.sqrt(3) / 2]]) + 0.01
    m = _dm_mesh(oracle_mod, pts)
    st = m.step()
    assert st["n_tri"] == 1
    # all l equal: fac_mu * mu = l, l0 = 1.2 l, f = 0.2 l, F_i = 0.6 (p_i - g)
    g = pts.mean(0)
    assert np.allclose(m.force(), 0.6 * (pts - g), rtol=0, atol=1e-15)
    m2 = _dm_mesh(oracle_mod, pts, fac_F=1.0)
    m2.step()
    assert np.abs(m2.force()).max() < 1e-15


def test_forces_sum_to_zero_and_fac_mu(oracle_mod):
    rng = np.random.default_rng(6)
    pts = rng.uniform(-0.5, 0.5, (300, 2))
    m = _dm_mesh(oracle_mod, pts)
    m.step()
    F = m.force()
    assert np.abs(F.sum(0)).max() < 1e-15 * m.fsum().sum() * 10
    # hexagon-shaped patch of the triangular lattice: every Delaunay edge has length s
    sp, R = 0.0390625, 5
    hexp = np.array([(i * sp + j * sp / 2, j * sp * math.sqrt(3) / 2)
                     for i in range(-R, R + 1) for j in range(-R, R + 1) if abs(i + j) <= R])
    sdf = W.grid_from_fn(lambda x, y: W.disk_sdf_fn(x, y, r=1.0), 128)
    mh = oracle_mod.OracleMesh(sdf, W.constant_grid(0.0390625), hexp, method=0, bounded=0, validity=0)
    st = mh.rebuild()
    assert st["fac_mu"] == pytest.approx(1.0, rel=1e-12)


@pytest.mark.parametrize("case", ["annulus_2e5", "disk_1e4"])
def test_fac_mu_sums_correctly_rounded(oracle_mod, case):
    """Eq. 3's sums: fac_mu equals sqrt of the ratio of correctly rounded
    sums (math.fsum) of l^2 and mu(m)^2 within a few ulps (the oracle sums
    pairwise).  A running sum drifts by 6e-15 over the annulus's 6e5 edges
    and by ~1e-13 over the disk's 3e4 identical mu^2 terms (uniform sizing:
    every rounding goes the same way); the comparison of forces near relaxed
    springs amplifies that."""
    if case == "disk_1e4":
        wl = W.disk_workload(n=10037, seed=0)
    else:
        wl = W.annulus_workload(n=200_003, seed=3, sdf_n=512, siz_n=256)
    om = oracle_mod.OracleMesh(wl.sdf, wl.sizing, wl.points, method=0)
    om.set_threads(4)
    st = om.rebuild()
    e, p = om.edges(), om.points()
    assert len(e) > (500_000 if case == "annulus_2e5" else 25_000)
    d = p[e[:, 1]] - p[e[:, 0]]
    l2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
    m = 0.5 * (p[e[:, 0]] + p[e[:, 1]])
    mu = W._bilinear_np(wl.sizing, m[:, 0], m[:, 1])
    want = math.sqrt(math.fsum(l2) / math.fsum(mu * mu))
    assert abs(st["fac_mu"] - want) <= 4e-16 * want, (st["fac_mu"] - want) / want


def test_quality_closed_forms(oracle_mod):
    eq = np.array([[0.0, 0.0], [0.05, 0.0], [0.025, 0.05 * math.sqrt(3) / 2]])
    st = _dm_mesh(oracle_mod, eq).rebuild()
    assert st["max_alpha"] == pytest.approx(1.0, rel=1e-12)
    assert st["max_beta"] == pytest.approx(1.0, rel=1e-12)
    assert st["min_angle_deg"] == pytest.approx(60.0, rel=1e-12)
    ri = np.array([[0.0, 0.0], [0.05, 0.0], [0.0, 0.05]])
    st = _dm_mesh(oracle_mod, ri).rebuild()
    assert st["max_alpha"] == pytest.approx((1 + math.sqrt(2)) / 2, rel=1e-12)
    assert st["max_beta"] == pytest.approx(math.sqrt(2), rel=1e-12)
    assert st["half_mean_alpha"] == pytest.approx((1 + math.sqrt(2)) / 2, rel=1e-12)


def _circle_mesh(oracle_mod, r=0.6):
    sdf = W.grid_from_fn(lambda x, y: W.disk_sdf_fn(x, y, r=r), 512)
    siz = W.constant_grid(1.0)
    pts = W.uniform_in(lambda x, y: W.disk_sdf_fn(x, y, r=r), 2000, 0)
    return oracle_mod.OracleMesh(sdf, siz, pts), r


def test_sphere_trace_hits_segment_crossing(oracle_mod):
    m, r = _circle_mesh(oracle_mod)
    rng = np.random.default_rng(7)
    cls, h, geps, havg = m.geometry()
    for _ in range(30):
        th = rng.uniform(0, 2 * np.pi)
        po = (r - 0.003) * np.array([math.cos(th), math.sin(th)])
        pn = po + 0.008 * np.array([math.cos(th + 0.3), math.sin(th + 0.3)])
        pf, c = m.project(po, 0, pn)
        # crossing of the segment with the circle
        d = (pn - po) / np.linalg.norm(pn - po)
        b = po @ d
        t = -b + math.sqrt(b * b - (po @ po - r * r))
        want = po + t * d
        assert c == 1
        assert np.linalg.norm(pf - want) < 2 * 0.01 * havg + 2e-5


def test_newton_projects_to_closest_point(oracle_mod):
    m, r = _circle_mesh(oracle_mod)
    rng = np.random.default_rng(8)
    cls, h, geps, havg = m.geometry()
    for _ in range(30):
        th = rng.uniform(0, 2 * np.pi)
        po = r * np.array([math.cos(th), math.sin(th)])
        pn = (r + 0.006) * np.array([math.cos(th + 0.01), math.sin(th + 0.01)])
        pf, c = m.project(po, 1, pn)
        want = r * pn / np.linalg.norm(pn)
        assert c == 1
        assert np.linalg.norm(pf - want) < 2 * 0.01 * havg + 2e-5


def test_geometry_counts_sum_to_n(oracle_mod):
    wa = W.annulus_workload(n=5000, sdf_n=128, siz_n=64)
    m = oracle_mod.OracleMesh(wa.sdf, wa.sizing, wa.points)
    cls, h, geps, havg = m.geometry()
    g = wa.sdf
    dx = (g.x1 - g.x0) / (g.nx - 1)
    dy = (g.y1 - g.y0) / (g.ny - 1)
    V = g.values.astype(np.float64)
    sm = 0.25 * (((V[:-1, :-1] + V[:-1, 1:]) + V[1:, :-1]) + V[1:, 1:])
    ldiag = math.hypot(dx, dy)
    want_cls = np.where(np.abs(sm) <= ldiag, 1, np.where(sm < 0, 0, 2))
    assert np.array_equal(cls, want_cls)
    sel = (cls == 0) | ((cls == 1) & (sm <= 0.5 * min(dx, dy)))
    # n^E_i = dx dy / h_i^2 sums to N over the selected cells
    assert (dx * dy / h[sel] ** 2).sum() == pytest.approx(5000, rel=1e-12)
    assert havg == pytest.approx(h[sel].mean(), rel=1e-12)
    assert np.allclose(geps, 0.01 * np.minimum(h, havg), rtol=1e-15)
