"""GPU parity of the automatic sizing pipeline (App. A, Sec. 3.3, Eq. 7) with
the oracle: medial points read off the device's triangles, and the whole
pipeline (samples, medial points, lfs, sizing grid) bit-identical."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

BOX = (-1.1, -1.1, 1.1, 1.1)


def test_medial_points_match():
    import paper_2309_13824_gb300 as g

    rng = np.random.default_rng(0)
    th = rng.uniform(0, 2 * np.pi, 3000)
    r = 0.8 + 0.05 * rng.standard_normal(3000)
    pts = np.stack([r * np.cos(th), r * np.sin(th)], 1)
    sdf = W.grid_from_fn(W.disk_sdf_fn, 129)
    siz = W.constant_grid(1.0)
    gm = g.Mesh(sdf, siz, pts, bounded=0, validity=0)
    gm.rebuild()
    vg, fg = gm.medial_points()
    om = oracle.OracleMesh(sdf, siz, pts, bounded=0, validity=0)
    om.rebuild()
    vo, fo = om.medial_points()
    assert np.array_equal(fg, fo)
    assert np.array_equal(vg[fg & 1 > 0, :2], vo[fo & 1 > 0, :2])
    assert np.array_equal(vg[fg & 2 > 0, 2:], vo[fo & 2 > 0, 2:])
    assert (fg & 2).astype(bool).sum() > 100


def _shapes():
    k = 200
    th = -2 * np.pi * np.arange(k) / k
    return {
        "square": np.array([[-0.5, -0.5], [-0.5, 0.5], [0.5, 0.5], [0.5, -0.5]]),
        "circle": 0.6 * np.stack([np.cos(th), np.sin(th)], 1),
        "rectangle": np.array([[-0.8, -0.1], [-0.8, 0.1], [0.8, 0.1], [0.8, -0.1]]),
        "star80": W.star_polygon(80, 0.4, 1.0, 9),
    }


@pytest.mark.parametrize("name", list(_shapes()))
def test_pipeline_matches(name):
    import paper_2309_13824_gb300 as g

    v = _shapes()[name]
    n, K = 129, 0.1
    sdf, mu, counts = g.auto_sizing(v, K, n, BOX)
    ref = oracle.auto_sizing(v, K, n, BOX)
    assert counts == {"samples": len(ref["samples"]), "medial": len(ref["medial"]), "kept": ref["kept"]}
    assert np.array_equal(sdf.view(np.uint32), ref["sdf"].view(np.uint32))
    want = ref["sizing"].astype(np.float32)
    assert np.array_equal(mu.view(np.uint32), want.view(np.uint32)), np.count_nonzero(mu != want)


def test_medial_points_of_a_cell_beyond_64_edges():
    """A point ringed by 70 others has a 70-edge cell: a capacity guard trip
    for the mesh, rebuilt in full for its medial points."""
    import ctypes as C

    import paper_2309_13824_gb300 as g
    from test_gpu_parity import _ringed_point

    sdf, siz, pts = _ringed_point(70)
    gm = g.Mesh(sdf, siz, pts, bounded=0, validity=0)
    st = g.mesh_stats()
    rc = g.lib().mesh_rebuild(gm._h, C.byref(st))
    assert rc == g.TRIME_EDEVICE and st.ring_overflow == 1 and st.exact_overflow == 0
    vg, fg = gm.medial_points()
    om = oracle.OracleMesh(sdf, siz, pts, bounded=0, validity=0)
    om.rebuild()
    vo, fo = om.medial_points()
    assert len(om.ring(0)) == 70 and fg[0] & 1
    assert np.array_equal(fg, fo)
    assert np.array_equal(vg[fg & 1 > 0, :2], vo[fo & 1 > 0, :2])
    assert np.array_equal(vg[fg & 2 > 0, 2:], vo[fo & 2 > 0, 2:])
