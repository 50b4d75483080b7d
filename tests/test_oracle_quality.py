"""Pins for the oracle's quality report (the statistics the paper tabulates
at termination, Sec. 5; alpha and beta of Sec. 3.6 Eqs. 11-12; the sizing
deviation of the valid edges, Eq. 3): closed forms of equilateral and right
isosceles triangles, and the order statistics, moments, shares and
histogram of a random mesh recomputed independently with numpy from the
textbook definitions alpha = R_circ / (2 r_in) (R = abc / 4A, r = A / s)."""
import math

import numpy as np
import pytest

import workloads as W


def _mesh(oracle_mod, pts, **kw):
    sdf = W.grid_from_fn(lambda x, y: W.disk_sdf_fn(x, y, r=1.0), 128)
    om = oracle_mod.OracleMesh(sdf, W.constant_grid(0.05), pts, method=0, **kw)
    om.rebuild()
    return om


def test_equilateral_patch(oracle_mod):
    sp, R = 0.0390625, 4
    hexp = np.array([(i * sp + j * sp / 2, j * sp * math.sqrt(3) / 2)
                     for i in range(-R, R + 1) for j in range(-R, R + 1) if abs(i + j) <= R])
    q = _mesh(oracle_mod, hexp, bounded=0, validity=0).quality()
    assert q["n_tri"] > 50
    for k in ("median_alpha", "mean_alpha", "max_alpha", "median_beta", "max_beta"):
        assert q[k] == pytest.approx(1.0, abs=1e-12), k
    assert q["std_alpha"] < 1e-12 and q["std_beta"] < 1e-12
    assert q["frac_alpha_lt_1_2"] == 1.0 and q["frac_alpha_lt_2"] == 1.0
    assert q["alpha_hist"][0] == q["n_tri"] and sum(q["alpha_hist"]) == q["n_tri"]
    assert q["min_angle_deg"] == pytest.approx(60.0, abs=1e-9)
    # every edge has the same length: fac_mu mu(m) = l, no deviation
    assert q["mean_size_dev"] < 1e-12 and q["p95_size_dev"] < 1e-12


def test_right_isosceles_pair(oracle_mod):
    # a square: two right isosceles triangles whichever diagonal SoS picks
    sq = np.array([[0.0, 0.0], [0.25, 0.0], [0.25, 0.25], [0.0, 0.25]])
    q = _mesh(oracle_mod, sq, bounded=0, validity=0).quality()
    assert q["n_tri"] == 2 and q["n_edges"] == 5
    a = (1 + math.sqrt(2)) / 2
    assert q["median_alpha"] == pytest.approx(a, rel=1e-14) and q["std_alpha"] < 1e-14
    assert q["median_beta"] == pytest.approx(math.sqrt(2), rel=1e-14)
    assert q["frac_alpha_lt_1_2"] == 0.0 and q["frac_alpha_lt_2"] == 1.0
    assert q["alpha_hist"] == [0, 0, 0, 2, 0, 0, 0, 0, 0, 0]  # [1.2, 1.3)
    assert q["min_angle_deg"] == pytest.approx(45.0, abs=1e-9)


@pytest.mark.parametrize("n", [3001, 3012])  # 3012 points: 8680 valid edges, 0.95 n an integer
def test_statistics_against_numpy(oracle_mod, n):
    wl = W.annulus_workload(n=n, seed=9, sdf_n=256, siz_n=128)
    om = oracle_mod.OracleMesh(wl.sdf, wl.sizing, wl.points, method=2)
    st = om.rebuild()
    q = om.quality()
    t, p, e = om.triangles(), om.points(), om.edges()
    A, B, Cc = p[t[:, 0]], p[t[:, 1]], p[t[:, 2]]
    a = np.linalg.norm(B - Cc, axis=1)
    b = np.linalg.norm(Cc - A, axis=1)
    c = np.linalg.norm(A - B, axis=1)
    area = 0.5 * np.abs((B - A)[:, 0] * (Cc - A)[:, 1] - (B - A)[:, 1] * (Cc - A)[:, 0])
    R = a * b * c / (4 * area)
    r = area / ((a + b + c) / 2)
    alpha = R / (2 * r)
    beta = np.maximum(np.maximum(a, b), c) / np.minimum(np.minimum(a, b), c)
    n = len(t)
    assert q["n_tri"] == n == st["n_tri"]
    assert q["n_edges"] % 20 or len(e) == 8680
    assert q["median_alpha"] == pytest.approx(np.sort(alpha)[(n - 1) // 2], rel=1e-12)
    assert q["median_beta"] == pytest.approx(np.sort(beta)[(n - 1) // 2], rel=1e-12)
    assert q["mean_alpha"] == pytest.approx(alpha.mean(), rel=1e-12)
    assert q["std_alpha"] == pytest.approx(alpha.std(), rel=1e-9)
    assert q["std_beta"] == pytest.approx(beta.std(), rel=1e-9)
    assert q["max_alpha"] == pytest.approx(alpha.max(), rel=1e-12)
    assert q["frac_alpha_lt_2"] == pytest.approx(np.mean(alpha < 2.0), abs=0.5 / n)
    edges = np.array([1.0, 1.05, 1.1, 1.2, 1.3, 1.5, 2.0, 3.0, 5.0, 10.0, np.inf])
    hist = np.histogram(np.maximum(alpha, 1.0), bins=edges)[0]
    assert np.abs(np.array(q["alpha_hist"]) - hist).sum() <= 2  # a value within rounding of an edge may move
    # smallest angle, law of cosines against arccos of the dot product
    ang = []
    for P0, P1, P2 in ((A, B, Cc), (B, Cc, A), (Cc, A, B)):
        u, v = P1 - P0, P2 - P0
        ang.append(np.degrees(np.arccos(np.clip((u * v).sum(1) / np.linalg.norm(u, axis=1) /
                                                np.linalg.norm(v, axis=1), -1, 1))))
    assert q["min_angle_deg"] == pytest.approx(np.min(ang), abs=1e-9)
    # sizing deviation over the valid edges, nearest-rank 95th percentile
    l = np.linalg.norm(p[e[:, 1]] - p[e[:, 0]], axis=1)
    m = 0.5 * (p[e[:, 0]] + p[e[:, 1]])
    mu = W._bilinear_np(wl.sizing, m[:, 0], m[:, 1])
    dev = np.abs(l / (st["fac_mu"] * mu) - 1)
    assert q["n_edges"] == len(e)
    assert q["mean_size_dev"] == pytest.approx(dev.mean(), rel=1e-12)
    k = math.ceil(0.95 * len(dev)) - 1
    assert q["p95_size_dev"] == pytest.approx(np.sort(dev)[k], rel=1e-12)
