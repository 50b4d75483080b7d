"""The device quality report (mesh_quality / mesh_batch_quality) against
the oracle's on the same rebuild: counts and histogram identical (a value
within rounding of a bin edge may move one count), order statistics,
maxima and means within 1e-12, standard deviations within 1e-9, shares
within one triangle; FP64 and FP32 positions (the oracle reads the same
float positions widened)."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import annulus_small, disk_small, make_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import oracle
    import paper_2309_13824_gb300 as g

    g.build()
    oracle.build()


def _same(qg, qo, precision=0):
    assert qg["n_tri"] == qo["n_tri"] and qg["n_edges"] == qo["n_edges"]
    n = max(qo["n_tri"], 1)
    assert np.abs(np.array(qg["alpha_hist"]) - np.array(qo["alpha_hist"])).sum() <= 2
    for k in ("median_alpha", "median_beta", "mean_alpha", "mean_beta", "max_alpha", "max_beta"):
        assert qg[k] == pytest.approx(qo[k], rel=1e-12, abs=1e-300), k
    for k in ("std_alpha", "std_beta"):
        assert qg[k] == pytest.approx(qo[k], rel=1e-9, abs=1e-15), k
    # fac_mu is the rebuild's own Eq. 3 factor: FP32 mode sums float terms,
    # so it and the sizing deviations built on it carry FP32 rounding
    tol = 1e-10 if precision == 0 else 2e-6
    for k in ("fac_mu", "mean_size_dev", "p95_size_dev"):
        assert qg[k] == pytest.approx(qo[k], rel=tol, abs=1e-15), k
    for k in ("frac_alpha_lt_1_2", "frac_alpha_lt_2"):
        assert abs(qg[k] - qo[k]) <= 1.0 / n, k
    assert qg["min_angle_deg"] == pytest.approx(qo["min_angle_deg"], abs=1e-9)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("which", ["disk", "annulus"])
def test_quality_report_matches_oracle(which, precision):
    wl = disk_small() if which == "disk" else annulus_small()
    gm, om = make_pair(wl, precision=precision, method=2)
    gm.rebuild()
    om.rebuild()
    _same(gm.quality(), om.quality(), precision)
    # after iterations: the report of a rebuild at the moved positions
    gm.step(5)
    P, cls, dp = gm.state()
    om.set_points(P.astype(np.float64))
    gm.rebuild()
    om.rebuild()
    qg = gm.quality()
    _same(qg, om.quality(), precision)
    assert qg["median_alpha"] < 1.3 and qg["n_tri"] > 1000


def test_quality_report_of_batch_meshes():
    import oracle
    import paper_2309_13824_gb300 as g

    meshes = [disk_small(n=3001, seed=4), annulus_small(n=5003, seed=6)]
    b = g.MeshBatch(meshes, method=2, autotune=False)
    b.rebuild()
    for k, (s, z, p) in enumerate(meshes):
        om = oracle.OracleMesh(s, z, p, method=2)
        om.rebuild()
        _same(b.quality(k), om.quality())


def test_quality_report_of_empty_mesh():
    import paper_2309_13824_gb300 as g

    sdf = W.grid_from_fn(lambda x, y: W.disk_sdf_fn(x, y, r=1.0), 64)
    m = g.Mesh(sdf, W.constant_grid(1.0), np.zeros((0, 2)))
    m.rebuild()
    q = m.quality()
    assert q["n_tri"] == 0 and q["n_edges"] == 0 and sum(q["alpha_hist"]) == 0
