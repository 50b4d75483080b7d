"""Pins of the oracle's point initialisation (Sec. 3.5): the counter-based
generator against its published reference outputs, the dithering's count
conservation and closeness to the expected counts, the density it follows,
and the projection of outside points."""
import numpy as np

import oracle as O
import workloads as W


def _square(n=65):
    return W.grid_from_fn(lambda x, y: np.maximum(np.abs(x), np.abs(y)) - 1.0, n)


def test_splitmix64_reference_outputs():
    # the first outputs of the SplitMix64 generator started from state 0
    assert [O.splitmix64(0, n) for n in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def _cells(grid, pts):
    dx = (grid.x1 - grid.x0) / (grid.values.shape[1] - 1)
    dy = (grid.y1 - grid.y0) / (grid.values.shape[0] - 1)
    i = np.clip(np.floor((pts[:, 0] - grid.x0) / dx), 0, grid.values.shape[1] - 2).astype(int)
    j = np.clip(np.floor((pts[:, 1] - grid.y0) / dy), 0, grid.values.shape[0] - 2).astype(int)
    return i, j


def test_uniform_square_counts():
    """Uniform density on the square: the dithered counts of the inner cells
    stay within one of the expected count, and the total is n_init up to the
    residuals the last cells cannot pass on."""
    sdf = _square(65)
    n_init = 20000
    p = O.init_points(sdf, W.constant_grid(1.0), n_init, seed=3)
    cls, h, geps, _ = O.OracleMesh(sdf, W.constant_grid(1.0), p[:10]).geometry()
    v = sdf.values.astype(np.float64)
    sm = 0.25 * (((v[:-1, :-1] + v[:-1, 1:]) + v[1:, :-1]) + v[1:, 1:])
    d = (sdf.x1 - sdf.x0) / (v.shape[1] - 1)
    sel = (cls == 0) | ((cls == 1) & (sm <= 0.5 * d))
    expect = n_init / sel.sum()
    assert abs(len(p) - n_init) <= 0.5 * sel.shape[1]
    i, j = _cells(sdf, p)
    counts = np.zeros(cls.shape, int)
    np.add.at(counts, (j, i), 1)
    assert np.abs(counts[cls == 0] - expect).max() < 1.5
    assert counts[~sel & (cls != 1)].sum() == 0  # nothing in outer cells


def test_density_follows_the_sizing_field():
    """The annulus sizing 0.002 + 0.05|sdf|: the share of points inside radius
    0.65 matches the share of the integral of 1/mu^2 there."""
    w = W.annulus_workload(n=1000, sdf_n=256, siz_n=128)
    p = O.init_points(w.sdf, w.sizing, 40000, seed=4)
    r = np.hypot(*p.T)
    share = np.mean(r < 0.65)
    rr = np.linspace(0.3, 1.0, 20001)
    mu = 0.002 + 0.05 * np.minimum(rr - 0.3, 1.0 - rr)
    f = rr / mu**2
    expect = np.trapezoid(f[rr < 0.65], rr[rr < 0.65]) / np.trapezoid(f, rr)
    assert abs(share - expect) < 0.02, (share, expect)


def test_points_inside_and_projected():
    w = W.annulus_workload(n=1000, sdf_n=256, siz_n=128)
    p = O.init_points(w.sdf, w.sizing, 30000, seed=5)
    s = W._bilinear_np(w.sdf, p[:, 0], p[:, 1])
    cls, h, geps, havg = O.OracleMesh(w.sdf, w.sizing, p[:10]).geometry()
    # the points generated outside were projected onto the boundary band
    assert np.all(s <= 2 * geps.max())
    assert np.mean(np.abs(s) <= geps.max()) > np.mean(s > 0)


def test_deterministic_and_seeded():
    sdf = _square(33)
    a = O.init_points(sdf, W.constant_grid(1.0), 3000, seed=7)
    b = O.init_points(sdf, W.constant_grid(1.0), 3000, seed=7)
    c = O.init_points(sdf, W.constant_grid(1.0), 3000, seed=8)
    assert np.array_equal(a, b) and len(a) == len(c) and not np.array_equal(a, c)
