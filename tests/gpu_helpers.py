"""Shared helpers of the GPU parity tests: build both implementations from the
same seeded workload and compare their results."""
import numpy as np

import oracle
import workloads as W

TOL_FP64 = 1e-12
TOL_FP32 = 2e-6


def sorted_tris(t):
    t = np.asarray(t, dtype=np.int64).reshape(-1, 3)
    if len(t) == 0:
        return t
    return t[np.lexsort((t[:, 2], t[:, 1], t[:, 0]))]


def make_pair(wl_or_args, precision=0, method=0, **params):
    """GPU mesh (debug recording on) and oracle mesh on identical inputs."""
    import paper_2309_13824_gb300 as g

    sdf, siz, pts = wl_or_args
    if precision == 1:
        pts = W.to_fp32_positions(pts)
    gm = g.Mesh(sdf, siz, pts, precision=precision, method=method, debug=1, **params)
    om = oracle.OracleMesh(sdf, siz, pts, method=method, **params)
    return gm, om


def h_of_points(om, pts):
    cls, h, geps, havg = om.geometry()
    out = np.empty(len(pts))
    for i, p in enumerate(pts):
        _, gi, gj = om.point_cell(float(p[0]), float(p[1]))
        out[i] = h[gj, gi]
    return out


def annulus_small(n=20011, seed=11, sdf_n=512, siz_n=256):
    wl = W.annulus_workload(n=n, seed=seed, sdf_n=sdf_n, siz_n=siz_n)
    return wl.sdf, wl.sizing, wl.points


def disk_small(n=10037, seed=0):
    wl = W.disk_workload(n=n, seed=seed)
    return wl.sdf, wl.sizing, wl.points
