"""Batched meshes (mesh_batch_*) vs the CPU oracle, mesh by mesh.

A batch steps several independent meshes with the same launches; per mesh
the result must be the one the oracle computes for that mesh alone:
identical triangle sets after a rebuild (whatever the bucket size and the
Voronoi lane count), and one-iteration moves within the FP64 / FP32
tolerances.  Meshes keep their own hybrid switch and termination.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import TOL_FP32, TOL_FP64, h_of_points, sorted_tris

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import paper_2309_13824_gb300 as g

    g.build()
    oracle.build()


def _mixed_meshes():
    """Uneven sizes and shapes: a disk, an annulus, a star whose size is a
    multiple of the 256-slot chunk, a 3-point mesh, an empty mesh, a square."""
    disk = W.grid_from_fn(W.disk_sdf_fn, 128)
    ann = W.grid_from_fn(W.annulus_sdf_fn, 256)
    ann_h = W.grid_from_fn(W.annulus_h_fn, 128)
    star_v = W.star_polygon(60, 0.4, 1.0, 21)
    star = W.polygon_sdf_grid(star_v, 256)
    star_h = W.Grid(np.ascontiguousarray(0.002 + 0.05 * np.abs(star.values), dtype=np.float32),
                    star.x0, star.y0, star.x1, star.y1)
    sq = W.grid_from_fn(W.square_sdf_fn, 128)

    def star_fn(x, y):
        return W._bilinear_np(star, x, y)

    return [
        (disk, W.constant_grid(0.01, 64), W.uniform_in(W.disk_sdf_fn, 1501, 31)),
        (ann, ann_h, W.density_in(W.annulus_sdf_fn, W.annulus_h_fn, 3001, 32)),
        (star, star_h, W.uniform_in(star_fn, 2048, 33)),
        (disk, W.constant_grid(0.01, 64), W.uniform_in(W.disk_sdf_fn, 3, 34)),
        (disk, W.constant_grid(0.01, 64), np.zeros((0, 2))),
        (sq, W.constant_grid(1.0), W.uniform_in(W.square_sdf_fn, 700, 35)),
    ]


def _fp(meshes, precision):
    if precision == 0:
        return meshes
    return [(s, z, W.to_fp32_positions(p)) for s, z, p in meshes]


def _oracles(meshes, **params):
    return [oracle.OracleMesh(s, z, p, **params) for s, z, p in meshes]


def _check_triangles(b, oms, stats):
    for k, om in enumerate(oms):
        om.rebuild()
        tg, to = sorted_tris(b.triangles(k)), sorted_tris(om.triangles())
        assert len(tg) == len(to), (k, len(tg), len(to))
        assert np.array_equal(tg, to), k
        assert stats[k]["n_tri"] == len(tg)
        assert stats[k]["ring_overflow"] == 0 and stats[k]["exact_overflow"] == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_triangles_match_oracle(precision):
    import paper_2309_13824_gb300 as g

    meshes = _fp(_mixed_meshes(), precision)
    b = g.MeshBatch(meshes, precision=precision, method=2, autotune=False)
    oms = _oracles(meshes, method=2)
    _check_triangles(b, oms, b.rebuild())
    # other tilings give the same triangles
    for n_opt, lanes in ((2.0, 32), (6.0, 16), (3.3, 32), (4.0, 8)):
        b.set_tuning(n_opt, lanes)
        assert b.tuning()["lanes"] == lanes
        _check_triangles(b, oms, b.rebuild())


def test_batch_autotune_record():
    import paper_2309_13824_gb300 as g

    meshes = _mixed_meshes()
    b = g.MeshBatch(meshes, method=2, autotune=True)
    t = b.tuning()
    assert len(t["candidates"]) == 9  # 3 bucket sizes x 8, 16, 32 lanes
    best = min(t["candidates"], key=lambda c: c[2])
    assert (t["n_opt"], t["lanes"]) == (best[0], best[1])
    assert t["n_slots"] == sum((len(m[2]) + 255) // 256 * 256 for m in meshes)
    _check_triangles(b, _oracles(meshes, method=2), b.rebuild())


@pytest.mark.parametrize("method,precision", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_batch_step_matches_oracle(method, precision):
    import paper_2309_13824_gb300 as g

    meshes = _fp(_mixed_meshes(), precision)
    b = g.MeshBatch(meshes, precision=precision, method=method, autotune=False)
    b.step(1)
    tol = TOL_FP64 if precision == 0 else TOL_FP32
    for k, (s, z, p) in enumerate(meshes):
        om = oracle.OracleMesh(s, z, p, method=method)
        om.step()
        pg, po = b.points(k).astype(np.float64), om.points()
        if len(po) == 0:
            continue
        if precision == 0:
            scale = h_of_points(om, po)
        else:
            scale = np.maximum(np.abs(po).max(1), 1e-3)
        err = np.linalg.norm(pg - po, axis=1) / scale
        bad = err > tol
        if precision == 0:
            assert bad.sum() == 0, (k, bad.sum(), err.max())
        else:
            assert bad.sum() <= max(2, 2e-3 * len(po)), (k, bad.sum(), err.max())


def test_batch_meshes_terminate_independently():
    import paper_2309_13824_gb300 as g

    meshes = _mixed_meshes()
    b = g.MeshBatch(meshes, method=2, autotune=False)
    st = b.step(400)
    iters = [s["iterations"] for s in st]
    live = [k for k, m in enumerate(meshes) if len(m[2]) > 3]
    assert all(st[k]["terminated"] for k in live), [s["terminated"] for s in st]
    assert len({iters[k] for k in live}) > 1, iters  # they stopped at different iterations
    # the same meshes stepped one at a time reach the same kind of end state
    for k in live:
        s, z, p = meshes[k]
        m = g.Mesh(s, z, p, method=2)
        sm = m.step(400)
        assert sm["terminated"]
        assert abs(sm["iterations"] - iters[k]) <= max(8, 0.3 * sm["iterations"]), (k, sm["iterations"], iters[k])
        assert st[k]["min_angle_deg"] == pytest.approx(sm["min_angle_deg"], abs=3.0)
        assert st[k]["half_mean_alpha"] == pytest.approx(sm["half_mean_alpha"], rel=2e-2)
    # finished meshes no longer move
    before = [b.points(k).copy() for k in range(len(meshes))]
    st2 = b.step(5)
    for k in live:
        assert np.array_equal(before[k], b.points(k))
        assert st2[k]["iterations"] == 0


def test_batch_set_state_resumes_one_mesh():
    import paper_2309_13824_gb300 as g

    meshes = _mixed_meshes()
    b = g.MeshBatch(meshes, method=0, autotune=False, fac_retria=0.0)
    b.step(3)
    k = 1
    s, z, p = meshes[k]
    om = oracle.OracleMesh(s, z, p, method=0, fac_retria=0.0)
    om.step()
    om.step()
    b.set_state(k, om.points(), om.classes(), om.dprev())
    b.set_method_state(k, 0)
    b.step(1)
    om.step()
    err = np.linalg.norm(b.points(k) - om.points(), axis=1) / h_of_points(om, om.points())
    assert err.max() < TOL_FP64


def test_batch_full_size_stars():
    # the 256-star batch of the benchmark (log-uniform 1e3..1e5 points, FP32
    # positions): complete triangle sets of the largest and of random meshes
    import os

    import paper_2309_13824_gb300 as g

    wl = W.star_batch_workload(workers=min(16, os.cpu_count() or 1))
    meshes = _fp(wl.meshes, 1)
    b = g.MeshBatch(meshes, precision=1, method=2, autotune=True)
    st = b.rebuild()
    assert sum(s["ring_overflow"] + s["exact_overflow"] for s in st) == 0
    sizes = np.array([len(m[2]) for m in meshes])
    rng = np.random.default_rng(0)
    pick = list(np.argsort(sizes)[-2:]) + list(rng.choice(len(meshes), 3, replace=False))
    for k in pick:
        s, z, p = meshes[k]
        om = oracle.OracleMesh(s, z, p, method=2)
        om.rebuild()
        tg, to = sorted_tris(b.triangles(int(k))), sorted_tris(om.triangles())
        assert np.array_equal(tg, to), int(k)
    b.step(3)
    assert all(s["n_tri"] > 0 for s in b.step(1))


def test_batch_distmesh_keeps_triangulations_per_mesh():
    # each mesh of a batch decides its own re-triangulations (Algorithm 1)
    import paper_2309_13824_gb300 as g

    # smooth shapes: the star's spike tips make unsynchronised trajectories
    # diverge exponentially (a projection near a corner amplifies rounding)
    mixed = _mixed_meshes()
    meshes = [mixed[0], mixed[1], mixed[5]]
    b = g.MeshBatch(meshes, method=0, autotune=False)
    oms = [oracle.OracleMesh(s, z, p, method=0) for s, z, p in meshes]
    kept = 0
    for step in range(40):
        st = b.step(1)
        for k, om in enumerate(oms):
            if st[k]["iterations"] == 0:
                continue  # this mesh has terminated
            so = om.step()
            assert st[k]["triangulations"] == so["triangulated"], (step, k)
            kept += 1 - so["triangulated"]
            err = np.linalg.norm(b.points(k) - om.points(), axis=1) / h_of_points(om, om.points())
            assert err.max() < 1e-6, (step, k, err.max())  # compounding step rounding
    assert kept > 0
