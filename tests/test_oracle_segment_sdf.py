"""Pins of the oracle's signed distance from clockwise line segments (Sec. 3.1)
against closed forms, an independent sampled builder and the sign rule's
corner cases."""
import numpy as np

import oracle as O
import workloads as W

SQUARE_CW = np.array([[0.0, 0.0], [0.0, 1.0], [1.0, 1.0], [1.0, 0.0]])


def _box_sdf(x, y):
    """Closed form for the unit square [0, 1]^2."""
    qx, qy = np.abs(x - 0.5) - 0.5, np.abs(y - 0.5) - 0.5
    outside = np.hypot(np.maximum(qx, 0), np.maximum(qy, 0))
    inside = np.minimum(np.maximum(qx, qy), 0)
    return outside + inside


def test_square_closed_form():
    rng = np.random.default_rng(0)
    x, y = rng.uniform(-1, 2, 5000), rng.uniform(-1, 2, 5000)
    s = O.segment_sdf(SQUARE_CW, x, y)
    assert np.allclose(s, _box_sdf(x, y), rtol=0, atol=1e-15)
    # an exact grid on the boundary and the vertices: zero
    assert np.all(O.segment_sdf(SQUARE_CW, [0, 0, 1, 1, 0.5, 0], [0, 1, 1, 0, 1, 0.25]) == 0)


def test_counter_clockwise_input_flips_the_sign():
    rng = np.random.default_rng(1)
    x, y = rng.uniform(-1, 2, 2000), rng.uniform(-1, 2, 2000)
    a = O.segment_sdf(SQUARE_CW, x, y)
    b = O.segment_sdf(SQUARE_CW[::-1], x, y)
    assert np.array_equal(a[a != 0], -b[a != 0])


def test_corner_signs():
    # L shape (clockwise): the reflex vertex (1, 1); points whose closest
    # point is a vertex take the sum of the two incident normals
    L_cw = np.array([[0, 0], [0, 2], [1, 2], [1, 1], [2, 1], [2, 0]], float)
    pts = np.array([
        [1.3, 1.3],    # outside, in the notch: the closest points lie on the two edges
        [0.9, 0.95],   # inside, closest to the reflex vertex (1, 1)
        [-0.2, -0.3],  # outside, closest to the convex corner (0, 0)
        [2.4, 1.3],    # outside, closest to the convex corner (2, 1)
        [0.1, 0.05],   # inside near the corner (0, 0), closest to the bottom edge
    ])
    s = O.segment_sdf(L_cw, pts[:, 0], pts[:, 1])
    expect = [0.3, -np.hypot(0.1, 0.05), np.hypot(0.2, 0.3), np.hypot(0.4, 0.3), -0.05]
    assert np.allclose(s, expect, rtol=0, atol=1e-15)


def test_star_against_sampled_builder():
    """The host builder of the workloads (nearest of dense samples, then its
    segment and neighbours; radial inside test) is an independent method: its
    distances are a minimum over a subset, so never below the oracle's, equal
    at almost every node, and the signs agree away from the boundary."""
    verts = W.star_polygon(300, 0.4, 1.0, 5)
    n = 129
    g = W.polygon_sdf_grid(verts, n)
    xs = g.x0 + np.arange(n) * ((g.x1 - g.x0) / (n - 1))
    ys = g.y0 + np.arange(n) * ((g.y1 - g.y0) / (n - 1))
    X, Y = np.meshgrid(xs, ys)
    s = O.segment_sdf(verts, X.ravel(), Y.ravel()).reshape(n, n)
    host = g.values.astype(np.float64)
    assert np.all(np.abs(host) >= np.abs(s).astype(np.float32).astype(np.float64) - 1e-7)
    same = np.abs(np.abs(host) - np.abs(s).astype(np.float32)) == 0
    assert same.mean() > 0.999
    far = np.abs(s) > 1e-6
    assert np.array_equal(np.sign(host[far]), np.sign(s[far]))


def test_regular_polygon_approaches_the_circle():
    k = 720
    th = -2 * np.pi * np.arange(k) / k  # clockwise
    verts = 0.8 * np.stack([np.cos(th), np.sin(th)], 1)
    rng = np.random.default_rng(2)
    x, y = rng.uniform(-1.5, 1.5, 3000), rng.uniform(-1.5, 1.5, 3000)
    s = O.segment_sdf(verts, x, y)
    circle = np.hypot(x, y) - 0.8
    sag = 0.8 * (1 - np.cos(np.pi / k))  # largest gap between polygon and circle
    assert np.all(np.abs(s - circle) <= sag + 1e-12)


def test_acute_tip_needs_the_summed_normal():
    """Just outside an acute tip, in its outer normal cone nearer the second
    segment's side: the first segment's normal alone would call the point
    inside; the sum of the two unit normals calls it outside."""
    tri_cw = np.array([[0.0, 0.0], [0.0, 1.0], [10.0, 0.5]])
    e1 = tri_cw[2] - tri_cw[1]
    e2 = tri_cw[0] - tri_cw[2]
    n1 = np.array([e1[1], -e1[0]]) / np.hypot(*e1)
    n2 = np.array([e2[1], -e2[0]]) / np.hypot(*e2)
    p = tri_cw[2] - (0.01 * n1 + 0.1 * n2)
    assert (p - tri_cw[2]) @ n1 > 0  # the single normal's verdict: inside
    s = O.segment_sdf(tri_cw, [p[0]], [p[1]])[0]
    assert s > 0 and np.isclose(s, np.hypot(*(p - tri_cw[2])), rtol=1e-14)
