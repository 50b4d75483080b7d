"""GPU parity of the Sec. 3.5 point initialisation (mesh_init_points) with the
oracle: the same points bit for bit, including the projected ones."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _cases():
    ann = W.annulus_workload(n=1000, sdf_n=256, siz_n=128)
    sq = W.grid_from_fn(lambda x, y: np.maximum(np.abs(x), np.abs(y)) - 1.0, 129)
    star = W.star_polygon(120, 0.4, 1.0, 3)
    star_sdf = W.polygon_sdf_grid(star, 257)
    star_siz = W.grid_from_fn(lambda x, y: 0.003 + 0.05 * np.hypot(x, y), 65)
    return {
        "annulus": (ann.sdf, ann.sizing, 30000),
        "square": (sq, W.constant_grid(1.0), 20000),
        "star": (star_sdf, star_siz, 25000),
    }


@pytest.mark.parametrize("name", list(_cases()))
def test_points_match(name):
    import paper_2309_13824_gb300 as g

    sdf, siz, n = _cases()[name]
    pg = g.init_points(sdf, siz, n, seed=11)
    po = oracle.init_points(sdf, siz, n, seed=11)
    assert pg.shape == po.shape
    assert np.array_equal(pg, po), np.count_nonzero(np.any(pg != po, 1))
    # some points were projected (they are not on their generating cell's uniform grid)
    s = W._bilinear_np(sdf, pg[:, 0], pg[:, 1])
    assert np.any(np.abs(s) < 1e-4)


def test_points_seed_a_mesh():
    """The initial points are a valid mesh_init input: the hybrid runs to
    termination from them."""
    import paper_2309_13824_gb300 as g

    ann = W.annulus_workload(n=1000, sdf_n=512, siz_n=256)
    p = g.init_points(ann.sdf, ann.sizing, 50000, seed=1)
    m = g.Mesh(ann.sdf, ann.sizing, p, method=2)
    s = m.step(500)
    assert s["terminated"] and s["min_angle_deg"] > 20


def test_polygon_to_mesh_input():
    """A spiky polygon all the way to a mesh: its automatic sizing (1024^2),
    10^5 initial points from it, and a mesh created and stepped from them."""
    import paper_2309_13824_gb300 as g

    box = (-1.1, -1.1, 1.1, 1.1)
    v = W.star_polygon(500, 0.4, 1.0, 2)
    sdf, mu, counts = g.auto_sizing(v, 0.1, 1024, box)
    sg, zg = W.Grid(sdf, *box), W.Grid(mu, *box)
    p = g.init_points(sg, zg, 100_000, seed=2)
    assert np.all(np.isfinite(p)) and np.all(np.abs(p) <= 1.1)
    m = g.Mesh(sg, zg, W.to_fp32_positions(p), method=2, precision=1)
    s = m.step(5, check=False)
    assert s["n_tri"] > 100_000
