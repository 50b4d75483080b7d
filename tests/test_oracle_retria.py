"""Re-triangulation skipping of the DistMesh method (Algorithm 1) in the
oracle: a step keeps the last triangulation exactly when no point has moved
more than fac_retria h_i since it was made, and the skipped steps move the
points by the springs of that triangulation's valid edges."""
import numpy as np

import oracle
import workloads as W


def _mesh(fac_retria, n=1500, seed=4):
    oracle.build()
    wl = W.disk_workload(n=n, seed=seed)
    return oracle.OracleMesh(wl.sdf, wl.sizing, wl.points, method=0, fac_retria=fac_retria), wl


def _h_at(om, p):
    cls, h, geps, havg = om.geometry()
    out = np.empty(len(p))
    for k, q in enumerate(p):
        _, gi, gj = om.point_cell(float(q[0]), float(q[1]))
        out[k] = h[gj, gi]
    return out


def test_every_step_triangulates_without_threshold():
    om, _ = _mesh(0.0)
    for _ in range(6):
        assert om.step()["triangulated"] == 1


def test_skip_rule_and_skipped_forces():
    om, _ = _mesh(0.1)
    tri_pos, tri_h, tri_edges = None, None, None
    skipped = 0
    expect = True  # the first step triangulates
    for it in range(40):
        p_before = om.points()
        st = om.step()
        if st["terminated"]:
            break
        assert bool(st["triangulated"]) == expect, it
        if st["triangulated"]:
            tri_pos, tri_h, tri_edges = p_before, _h_at(om, p_before), om.edges()
        else:
            skipped += 1
            # the rule: no point was farther than 0.1 h_i from its triangulated position
            assert np.all(np.linalg.norm(p_before - tri_pos, axis=1) <= 0.1 * tri_h)
            # the springs of the kept valid edges, recomputed here from the positions
            assert np.array_equal(om.edges(), tri_edges)
            e = tri_edges
            d = p_before[e[:, 0]] - p_before[e[:, 1]]
            ln = np.linalg.norm(d, axis=1)
            mid = 0.5 * (p_before[e[:, 0]] + p_before[e[:, 1]])
            mu = np.array([oracle.bilinear(W.constant_grid(0.01, 256), x, y) for x, y in mid])
            fac = np.sqrt((ln**2).sum() / (mu**2).sum())
            l0 = 1.2 * fac * mu
            f = np.where(ln < l0, l0 - ln, 0.0)
            F = np.zeros_like(p_before)
            np.add.at(F, e[:, 0], (f / ln)[:, None] * d)
            np.add.at(F, e[:, 1], -(f / ln)[:, None] * d)
            scale = np.zeros(len(F))
            np.add.at(scale, e[:, 0], ln)
            np.add.at(scale, e[:, 1], ln)
            assert np.all(np.linalg.norm(om.force() - F, axis=1) <= 1e-12 * np.maximum(scale, 1e-300))
        # the next step re-triangulates iff some point is now farther than 0.1 h_i
        expect = bool(np.any(np.linalg.norm(om.points() - tri_pos, axis=1) > 0.1 * tri_h))
    assert skipped > 0


def test_skipping_reaches_the_same_quality():
    def run(fac):
        om, _ = _mesh(fac, n=1200, seed=6)
        tri = 0
        st = None
        for _ in range(300):
            st = om.step()
            tri += st["triangulated"]
            if st["terminated"]:
                break
        return st, tri

    s0, t0 = run(0.0)
    s1, t1 = run(0.1)
    assert t1 < t0
    assert abs(s1["half_mean_alpha"] - s0["half_mean_alpha"]) < 0.02 * s0["half_mean_alpha"]
