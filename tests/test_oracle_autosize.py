"""Pins of the oracle's automatic sizing pipeline (App. A boundary samples,
Sec. 3.3 medial axis and local feature size) against shapes whose medial
axis is known in closed form."""
import numpy as np
from scipy.spatial import cKDTree

import oracle as O


def _square(side=1.0):
    h = side / 2
    return np.array([[-h, -h], [-h, h], [h, h], [h, -h]])  # clockwise


def _regular(k, r):
    th = -2 * np.pi * np.arange(k) / k
    return r * np.stack([np.cos(th), np.sin(th)], 1)


def test_samples_lie_on_the_boundary_and_are_spaced():
    v = _regular(60, 0.7)
    ds, ge = 0.03, 3e-4
    S = O.boundary_samples(v, ds, ge)
    assert np.all(np.abs(O.segment_sdf(v, S[:, 0], S[:, 1])) <= ge)
    d, _ = cKDTree(S).query(S, k=2)
    assert d[:, 1].min() >= ds
    # no hole: consecutive samples along the loop are less than 2 ds apart
    ang = np.sort(np.arctan2(S[:, 1], S[:, 0]))
    gaps = np.diff(np.concatenate([ang, ang[:1] + 2 * np.pi])) * 0.7
    assert gaps.max() < 2 * ds * 1.05


def test_thin_strip_keeps_both_sides():
    # 1 x 0.01 strip, samples 0.02 apart: the two long sides are closer than
    # ds but their midpoints are not on the boundary, so neither side is merged away
    w = 0.01
    strip = np.array([[-0.5, -w / 2], [-0.5, w / 2], [0.5, w / 2], [0.5, -w / 2]])
    S = O.boundary_samples(strip, 0.02, 1e-4)
    top, bottom = np.sum(np.isclose(S[:, 1], w / 2)), np.sum(np.isclose(S[:, 1], -w / 2))
    assert top >= 20 and bottom >= 20


def test_square_lfs_is_the_distance_to_the_diagonals():
    r = O.auto_sizing(_square(1.0), 0.1, 129)
    S, lf, ds = r["samples"], r["lfs"], r["ds"]
    true = np.minimum(np.abs(S[:, 0] - S[:, 1]), np.abs(S[:, 0] + S[:, 1])) / np.sqrt(2)
    assert np.all(np.abs(lf - true) <= 3 * ds), np.abs(lf - true).max()
    # Eq. 7 on the samples: never above lfs
    assert np.all(O.sizing_field(S, lf, 0.1, S[:, 0], S[:, 1]) <= lf)


def test_circle_lfs_is_the_radius():
    r = O.auto_sizing(_regular(400, 0.5), 0.1, 129)
    # the kept medial points gather at the centre, none near the boundary
    assert np.all(np.abs(r["lfs"] - 0.5) <= 3 * r["ds"]), np.abs(r["lfs"] - 0.5).max()


def test_narrow_rectangle_lfs_is_half_the_width():
    w = 0.2
    rect = np.array([[-0.8, -w / 2], [-0.8, w / 2], [0.8, w / 2], [0.8, -w / 2]])
    r = O.auto_sizing(rect, 0.1, 129)
    S, lf = r["samples"], r["lfs"]
    mid = (np.abs(S[:, 0]) < 0.5) & (np.abs(np.abs(S[:, 1]) - w / 2) < 1e-12)
    assert mid.sum() > 20
    assert np.all(np.abs(lf[mid] - w / 2) <= 2 * r["ds"])


def test_isolated_medial_points_are_trimmed():
    rng = np.random.default_rng(0)
    cluster = rng.normal(0, 0.01, (50, 2))
    lone = np.array([[0.9, 0.9]])
    M = np.concatenate([cluster, lone])
    S = np.array([[0.9, 0.95], [0.0, 0.1]])
    lf, kept = O.lfs(S, M, 0.06, 3)
    assert kept == 50
    assert np.isclose(lf[0], np.min(np.hypot(*(cluster - S[0]).T)))  # the lone point no longer counts
    # nothing kept: every point counts
    lf2, kept2 = O.lfs(S, lone, 0.06, 3)
    assert kept2 == 0 and np.isclose(lf2[0], 0.05)
