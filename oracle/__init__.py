"""ctypes front end of the plain FP64 CPU oracle (TriMe++, arXiv 2309.13824).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package.  The
product path must never route through it.  It shares no code with the CUDA
library; the only common dependency is the seeded input generator module
``workloads``.

``build()`` compiles ``trime_oracle.c`` with ``-O2 -ffp-contract=off`` (the
fixed floating-point formulas of the triangle-set definition must not be
contracted into FMAs) into ``oracle/_build/libtrime_oracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "trime_oracle.c"
_HDR = _HERE / "trime_oracle.h"
_OUT = _HERE / "_build" / "libtrime_oracle.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle shared library (gcc, no FMA contraction)."""
    _OUT.parent.mkdir(exist_ok=True)
    if force or not _OUT.exists() or _OUT.stat().st_mtime < max(_SRC.stat().st_mtime, _HDR.stat().st_mtime):
        tmp = _OUT.with_suffix(f".{os.getpid()}.tmp")
        cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-o", str(tmp), str(_SRC), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("x0", C.c_double), ("y0", C.c_double),
                ("x1", C.c_double), ("y1", C.c_double), ("v", C.POINTER(C.c_float))]


class _Params(C.Structure):
    _fields_ = [("method", C.c_int32), ("bounded", C.c_int32), ("validity", C.c_int32),
                ("newton_max", C.c_int32), ("trace_max", C.c_int32), ("quad_max_level", C.c_int32),
                ("fac_F", C.c_double), ("k_spring", C.c_double), ("dt", C.c_double),
                ("fac_pt", C.c_double), ("fac_geps", C.c_double), ("fac_voro_bound", C.c_double),
                ("fac_end", C.c_double), ("T_circ", C.c_double), ("T_switch", C.c_double),
                ("T_end_q", C.c_double), ("T_end_amax", C.c_double), ("N_opt", C.c_double),
                ("eta", C.c_double), ("damping", C.c_double), ("fac_retria", C.c_double),
                ("fac_add", C.c_double), ("T_add", C.c_double), ("n_total", C.c_int64)]


class _Stats(C.Structure):
    _fields_ = [("n_tri", C.c_int64), ("n_edges", C.c_int64), ("half_mean_alpha", C.c_double),
                ("half_mean_beta", C.c_double), ("max_alpha", C.c_double), ("max_beta", C.c_double),
                ("min_angle_deg", C.c_double), ("mean_size_dev", C.c_double), ("fac_mu", C.c_double),
                ("newton_fail", C.c_int64), ("trace_cap", C.c_int64), ("quad_cap", C.c_int64),
                ("clip_errors", C.c_int64), ("method_used", C.c_int32), ("terminated", C.c_int32),
                ("switched", C.c_int32), ("small_moves", C.c_int32), ("triangulated", C.c_int32),
                ("added", C.c_int64), ("n_points", C.c_int64)]


class _Quality(C.Structure):
    _fields_ = [("n_tri", C.c_int64), ("n_edges", C.c_int64), ("median_alpha", C.c_double),
                ("median_beta", C.c_double), ("mean_alpha", C.c_double), ("mean_beta", C.c_double),
                ("max_alpha", C.c_double), ("max_beta", C.c_double), ("std_alpha", C.c_double),
                ("std_beta", C.c_double), ("frac_alpha_lt_1_2", C.c_double), ("frac_alpha_lt_2", C.c_double),
                ("min_angle_deg", C.c_double), ("alpha_hist", C.c_int64 * 10), ("fac_mu", C.c_double),
                ("mean_size_dev", C.c_double), ("p95_size_dev", C.c_double)]


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(str(build()))
        P = C.POINTER
        dp, ip, u8p, i64p = P(C.c_double), P(C.c_int32), P(C.c_uint8), P(C.c_int64)
        lib.om_default_params.argtypes = [P(_Params)]
        lib.om_create.restype = C.c_void_p
        lib.om_create.argtypes = [P(_Grid), P(_Grid), dp, C.c_int64, P(_Params)]
        lib.om_destroy.argtypes = [C.c_void_p]
        lib.om_last_error.restype = C.c_char_p
        for name in ("om_rebuild", "om_step"):
            getattr(lib, name).argtypes = [C.c_void_p]
        lib.om_rebuild_sample.argtypes = [C.c_void_p, i64p, C.c_int64, C.c_int]
        lib.om_set_threads.argtypes = [C.c_void_p, C.c_int]
        lib.om_quality_report.argtypes = [C.c_void_p, C.POINTER(_Quality)]
        lib.om_quality_report.restype = None
        lib.om_rebuild_sample_mt.restype = C.c_int64
        lib.om_rebuild_sample_mt.argtypes = [C.c_void_p, i64p, C.c_int64, C.c_int, C.c_int]
        lib.om_sample_triangles.restype = C.c_int64
        lib.om_sample_triangles.argtypes = [C.c_void_p, i64p, C.c_int64, ip, C.c_int64]
        for name in ("om_num_points", "om_num_triangles", "om_num_edges"):
            getattr(lib, name).restype = C.c_int64
            getattr(lib, name).argtypes = [C.c_void_p]
        lib.om_get_triangles.argtypes = [C.c_void_p, ip]
        lib.om_get_edges.argtypes = [C.c_void_p, ip]
        for name in ("om_get_points", "om_set_points", "om_get_dprev", "om_set_dprev", "om_get_pnew",
                     "om_get_force", "om_get_fsum", "om_get_centroid", "om_get_cell_area"):
            getattr(lib, name).argtypes = [C.c_void_p, dp]
        lib.om_get_class.argtypes = [C.c_void_p, u8p]
        lib.om_set_class.argtypes = [C.c_void_p, u8p]
        lib.om_get_quad_level.argtypes = [C.c_void_p, ip]
        lib.om_get_stats.argtypes = [C.c_void_p, P(_Stats)]
        lib.om_set_method_state.argtypes = [C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_double]
        lib.om_get_ring.argtypes = [C.c_void_p, C.c_int64, ip, C.c_int]
        lib.om_get_cell_polygon.argtypes = [C.c_void_p, C.c_int64, dp, C.c_int]
        lib.om_get_geometry.argtypes = [C.c_void_p, u8p, dp, dp, dp]
        lib.om_point_cell.argtypes = [C.c_void_p, C.c_double, C.c_double, ip, ip]
        lib.om_orient2d.argtypes = [dp, dp, dp]
        lib.om_incircle.argtypes = [dp, dp, dp, dp]
        lib.om_incircle_sos.argtypes = [dp, C.c_int64, dp, C.c_int64, dp, C.c_int64, dp, C.c_int64]
        lib.om_bilinear.restype = C.c_double
        lib.om_bilinear.argtypes = [P(_Grid), C.c_double, C.c_double]
        lib.om_polygon_centroid.argtypes = [P(_Grid), dp, dp, C.c_int, C.c_double, C.c_int, dp, ip]
        lib.om_project_point.argtypes = [C.c_void_p, dp, C.c_int, dp, dp, ip]
        lib.om_segment_sdf.argtypes = [dp, C.c_int64, dp, dp, C.c_int64, dp]
        lib.om_sizing_field.argtypes = [dp, dp, C.c_int64, C.c_double, dp, dp, C.c_int64, dp]
        lib.om_boundary_samples.restype = C.c_int64
        lib.om_boundary_samples.argtypes = [dp, C.c_int64, C.c_double, C.c_double, dp, C.c_int64]
        lib.om_medial_points.argtypes = [C.c_void_p, dp, u8p]
        lib.om_init_points.restype = C.c_int64
        lib.om_init_points.argtypes = [P(_Grid), P(_Grid), C.c_int64, C.c_uint64, P(_Params), dp, C.c_int64]
        lib.om_splitmix64.restype = C.c_uint64
        lib.om_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        lib.om_lfs.restype = C.c_int64
        lib.om_lfs.argtypes = [dp, C.c_int64, dp, C.c_int64, C.c_double, C.c_int32, dp]
        lib.om_adf_build.restype = C.c_void_p
        lib.om_adf_build.argtypes = [dp, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32,
                                     C.c_int32, ip, dp, C.c_int32, C.c_int32]
        lib.om_adf_size.restype = C.c_int64
        lib.om_adf_size.argtypes = [C.c_void_p]
        lib.om_adf_export.argtypes = [C.c_void_p, dp, ip, ip, ip]
        lib.om_adf_eval.argtypes = [C.c_void_p, dp, dp, C.c_int64, dp]
        lib.om_adf_free.argtypes = [C.c_void_p]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _cgrid(g):
    v = np.ascontiguousarray(g.values, dtype=np.float32)
    cg = _Grid(g.nx, g.ny, g.x0, g.y0, g.x1, g.y1, v.ctypes.data_as(C.POINTER(C.c_float)))
    return cg, v


PARAM_DEFAULTS = None


def default_params() -> dict:
    lib = _load()
    p = _Params()
    lib.om_default_params(C.byref(p))
    return {name: getattr(p, name) for name, _ in _Params._fields_}


def _pt(p):
    return np.ascontiguousarray(p, dtype=np.float64).reshape(-1)


def orient2d(a, b, c) -> int:
    return _load().om_orient2d(_dp(_pt(a)), _dp(_pt(b)), _dp(_pt(c)))


def incircle(a, b, c, d) -> int:
    return _load().om_incircle(_dp(_pt(a)), _dp(_pt(b)), _dp(_pt(c)), _dp(_pt(d)))


def incircle_sos(a, ia, b, ib, c, ic, d, idd) -> int:
    return _load().om_incircle_sos(_dp(_pt(a)), ia, _dp(_pt(b)), ib, _dp(_pt(c)), ic, _dp(_pt(d)), idd)


def bilinear(grid, x, y) -> float:
    cg, keep = _cgrid(grid)
    return _load().om_bilinear(C.byref(cg), float(x), float(y))


def polygon_centroid(sizing, gen, poly, eps_c, max_level=8):
    cg, keep = _cgrid(sizing)
    c = np.zeros(2)
    lv = C.c_int32()
    poly = np.ascontiguousarray(poly, dtype=np.float64)
    _load().om_polygon_centroid(C.byref(cg), _dp(_pt(gen)), _dp(poly), len(poly), eps_c, max_level, _dp(c),
                                C.byref(lv))
    return c, lv.value


def segment_sdf(verts_cw, px, py) -> np.ndarray:
    """Sec. 3.1 SDF of the clockwise loop verts_cw (n, 2) at the points
    (px, py), FP64, brute force (see om_segment_sdf)."""
    lib = _load()
    v = np.ascontiguousarray(verts_cw, dtype=np.float64).reshape(-1, 2)
    px = np.ascontiguousarray(px, dtype=np.float64).ravel()
    py = np.ascontiguousarray(py, dtype=np.float64).ravel()
    out = np.empty(len(px))
    if lib.om_segment_sdf(_dp(v), len(v), _dp(px), _dp(py), len(px), _dp(out)) != 0:
        raise ValueError(lib.om_last_error().decode())
    return out


class OracleADF:
    """Sec. 3.7 adaptive distance field of the clockwise loop verts_cw: one
    quadtree per listed cell (index j (nx - 1) + i of the node grid over box),
    split while the bilinear error at the edge midpoints and the centre
    exceeds tol[r] and the level is below max_depth (om_adf_build)."""

    def __init__(self, verts_cw, box, nx, ny, cells, tol, max_depth=10):
        lib = _load()
        self._v = np.ascontiguousarray(verts_cw, dtype=np.float64).reshape(-1, 2)
        c = np.ascontiguousarray(cells, dtype=np.int32).ravel()
        t = np.ascontiguousarray(tol, dtype=np.float64).ravel()
        x0, y0, x1, y1 = (float(b) for b in box)
        self._h = lib.om_adf_build(_dp(self._v), len(self._v), x0, y0, x1, y1, int(nx), int(ny),
                                   c.ctypes.data_as(C.POINTER(C.c_int32)), _dp(t), len(c), int(max_depth))
        if not self._h:
            raise ValueError(lib.om_last_error().decode())

    def nodes(self):
        """(v (n, 4), child (n,), root (n,), lev (n, 3)) in build order."""
        lib = _load()
        n = lib.om_adf_size(self._h)
        v = np.zeros((n, 4))
        child = np.zeros(n, np.int32)
        root = np.zeros(n, np.int32)
        lev = np.zeros((n, 3), np.int32)
        ip = C.POINTER(C.c_int32)
        lib.om_adf_export(self._h, _dp(v), child.ctypes.data_as(ip), root.ctypes.data_as(ip), lev.ctypes.data_as(ip))
        return v, child, root, lev

    def eval(self, px, py):
        lib = _load()
        px = np.ascontiguousarray(px, dtype=np.float64).ravel()
        py = np.ascontiguousarray(py, dtype=np.float64).ravel()
        out = np.empty(len(px))
        lib.om_adf_eval(self._h, _dp(px), _dp(py), len(px), _dp(out))
        return out

    def __del__(self):
        if getattr(self, "_h", None):
            _load().om_adf_free(self._h)
            self._h = None


def sizing_field(samples, lfs, K, px, py) -> np.ndarray:
    """Eq. 7: min over the samples of K |s - x| + lfs(s) at the points
    (px, py), FP64, brute force (om_sizing_field)."""
    lib = _load()
    s = np.ascontiguousarray(samples, dtype=np.float64).reshape(-1, 2)
    lf = np.ascontiguousarray(lfs, dtype=np.float64).ravel()
    px = np.ascontiguousarray(px, dtype=np.float64).ravel()
    py = np.ascontiguousarray(py, dtype=np.float64).ravel()
    out = np.empty(len(px))
    if lib.om_sizing_field(_dp(s), _dp(lf), len(s), float(K), _dp(px), _dp(py), len(px), _dp(out)) != 0:
        raise ValueError(lib.om_last_error().decode())
    return out


def boundary_samples(verts_cw, ds, geps_hat) -> np.ndarray:
    """App. A boundary samples of a clockwise segment loop, trimmed (om_boundary_samples)."""
    lib = _load()
    v = np.ascontiguousarray(verts_cw, dtype=np.float64).reshape(-1, 2)
    n = lib.om_boundary_samples(_dp(v), len(v), float(ds), float(geps_hat), None, 0)
    if n < 0:
        raise ValueError(lib.om_last_error().decode())
    out = np.empty((n, 2))
    lib.om_boundary_samples(_dp(v), len(v), float(ds), float(geps_hat), _dp(out), n)
    return out


def init_points(sdf, sizing, n_init, seed=0, **params) -> np.ndarray:
    """Sec. 3.5 initial points (om_init_points), (n, 2) float64."""
    lib = _load()
    p = _Params()
    lib.om_default_params(C.byref(p))
    for k, v in params.items():
        setattr(p, k, v)
    gs, gz = _cgrid(sdf), _cgrid(sizing)
    n = lib.om_init_points(C.byref(gs[0]), C.byref(gz[0]), int(n_init), int(seed), C.byref(p), None, 0)
    if n < 0:
        raise ValueError(lib.om_last_error().decode())
    out = np.empty((n, 2))
    lib.om_init_points(C.byref(gs[0]), C.byref(gz[0]), int(n_init), int(seed), C.byref(p), _dp(out), n)
    return out


def splitmix64(seed, n) -> int:
    return int(_load().om_splitmix64(seed, n))


def lfs(samples, medial, r_nei, n_thres=3):
    """Trimmed medial points and the local feature size of every sample (om_lfs):
    (lfs (ns,), number of medial points kept)."""
    lib = _load()
    s = np.ascontiguousarray(samples, dtype=np.float64).reshape(-1, 2)
    m = np.ascontiguousarray(medial, dtype=np.float64).reshape(-1, 2)
    out = np.empty(len(s))
    kept = lib.om_lfs(_dp(s), len(s), _dp(m), len(m), float(r_nei), int(n_thres), _dp(out))
    if kept < 0:
        raise ValueError(lib.om_last_error().decode())
    return out, int(kept)


def medial_list(v, flags) -> np.ndarray:
    """The medial points in sample order, v1 then v2 of each sample."""
    pts = []
    for i in range(len(flags)):
        if flags[i] & 1:
            pts.append(v[i, :2])
        if flags[i] & 2:
            pts.append(v[i, 2:])
    return np.array(pts).reshape(-1, 2)


def auto_sizing(verts_cw, K, n, box=(-1.1, -1.1, 1.1, 1.1), fac_s=0.5, fac_geps=0.01, fac_nei=2.0, n_thres=3):
    """The automatic sizing pipeline (App. A, Sec. 3.3, Eq. 7) on an n x n node
    grid over box: boundary samples, their Delaunay triangles (unbounded cells,
    no validity tests) on the oracle's own SDF grid, medial points, lfs, and
    the sizing field at the nodes (FP64)."""
    x0, y0, x1, y1 = box
    dx, dy = (x1 - x0) / (n - 1), (y1 - y0) / (n - 1)
    g = min(dx, dy)
    ds, geps_hat = fac_s * g, fac_geps * g
    S = boundary_samples(verts_cw, ds, geps_hat)
    xs = x0 + np.arange(n) * dx
    ys = y0 + np.arange(n) * dy
    X, Y = np.meshgrid(xs, ys)
    sdf = segment_sdf(verts_cw, X.ravel(), Y.ravel()).reshape(n, n).astype(np.float32)
    from workloads import Grid, constant_grid

    om = OracleMesh(Grid(sdf, x0, y0, x1, y1), constant_grid(1.0, 2, box), S, bounded=0, validity=0)
    om.rebuild()
    v, flags = om.medial_points()
    M = medial_list(v, flags)
    lf, kept = lfs(S, M, fac_nei * n_thres * ds, n_thres)
    mu = sizing_field(S, lf, K, X.ravel(), Y.ravel()).reshape(n, n)
    return {"samples": S, "medial": M, "kept": kept, "lfs": lf, "sizing": mu, "sdf": sdf, "ds": ds}


class OracleMesh:
    """One mesh in the oracle; positions are float64 (FP32-mode inputs are
    passed already widened)."""

    def __init__(self, sdf, sizing, xy, **params):
        lib = _load()
        self._lib = lib
        p = _Params()
        lib.om_default_params(C.byref(p))
        for k, v in params.items():
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, v)
        self.params = p
        self._sdf = _cgrid(sdf)
        self._siz = _cgrid(sizing)
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        h = lib.om_create(C.byref(self._sdf[0]), C.byref(self._siz[0]), _dp(xy), len(xy), C.byref(p))
        if not h:
            raise ValueError(lib.om_last_error().decode())
        self._h = h
        self.ncx, self.ncy = sdf.nx - 1, sdf.ny - 1

    @property
    def n(self) -> int:
        """N_current (grows under the point-addition scheme)."""
        return int(self._lib.om_num_points(self._h))

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.om_destroy(self._h)
            self._h = None

    def set_threads(self, threads: int):
        """OpenMP threads for the per-cell loops of rebuild()/step() (results
        are those of one thread)."""
        self._lib.om_set_threads(self._h, int(threads))

    def rebuild(self):
        self._lib.om_rebuild(self._h)
        return self.stats()

    def step(self):
        self._lib.om_step(self._h)
        return self.stats()

    def rebuild_sample(self, cells, with_centroid: bool = True):
        """Procedure I on the given cells (and their CVD centroids), single thread."""
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        self._lib.om_rebuild_sample(self._h, cells.ctypes.data_as(C.POINTER(C.c_int64)), len(cells),
                                    int(with_centroid))

    def rebuild_sample_mt(self, cells, with_centroid: bool = True, threads: int = 0) -> int:
        """rebuild_sample's work on `threads` OpenMP threads (0: all cores); timing only."""
        import os

        cells = np.ascontiguousarray(cells, dtype=np.int64)
        nt = threads or (os.cpu_count() or 1)
        return self._lib.om_rebuild_sample_mt(self._h, cells.ctypes.data_as(C.POINTER(C.c_int64)), len(cells),
                                              int(with_centroid), nt)

    def sample_triangles(self, cells) -> np.ndarray:
        """Valid triangles owned (smallest index) by the given cells."""
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        cp = cells.ctypes.data_as(C.POINTER(C.c_int64))
        n = self._lib.om_sample_triangles(self._h, cp, len(cells), None, 0)
        t = np.zeros((n, 3), dtype=np.int32)
        if n:
            self._lib.om_sample_triangles(self._h, cp, len(cells), t.ctypes.data_as(C.POINTER(C.c_int32)), n)
        return t

    def stats(self) -> dict:
        s = _Stats()
        self._lib.om_get_stats(self._h, C.byref(s))
        return {name: getattr(s, name) for name, _ in _Stats._fields_}

    def quality(self) -> dict:
        """om_quality_report of the last rebuild (at the current positions)."""
        q = _Quality()
        self._lib.om_quality_report(self._h, C.byref(q))
        d = {name: getattr(q, name) for name, _ in _Quality._fields_}
        d["alpha_hist"] = list(q.alpha_hist)
        return d

    def triangles(self) -> np.ndarray:
        n = self._lib.om_num_triangles(self._h)
        t = np.zeros((n, 3), dtype=np.int32)
        if n:
            self._lib.om_get_triangles(self._h, t.ctypes.data_as(C.POINTER(C.c_int32)))
        return t

    def edges(self) -> np.ndarray:
        n = self._lib.om_num_edges(self._h)
        e = np.zeros((n, 2), dtype=np.int32)
        if n:
            self._lib.om_get_edges(self._h, e.ctypes.data_as(C.POINTER(C.c_int32)))
        return e

    def _get2(self, fn):
        a = np.zeros((self.n, 2))
        getattr(self._lib, fn)(self._h, _dp(a))
        return a

    def _get1(self, fn):
        a = np.zeros(self.n)
        getattr(self._lib, fn)(self._h, _dp(a))
        return a

    def points(self):
        return self._get2("om_get_points")

    def set_points(self, xy):
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        self._lib.om_set_points(self._h, _dp(xy))

    def pnew(self):
        return self._get2("om_get_pnew")

    def force(self):
        return self._get2("om_get_force")

    def fsum(self):
        return self._get1("om_get_fsum")

    def centroid(self):
        return self._get2("om_get_centroid")

    def cell_area(self):
        return self._get1("om_get_cell_area")

    def dprev(self):
        return self._get1("om_get_dprev")

    def set_dprev(self, d):
        d = np.ascontiguousarray(d, dtype=np.float64)
        self._lib.om_set_dprev(self._h, _dp(d))

    def classes(self):
        c = np.zeros(self.n, dtype=np.uint8)
        self._lib.om_get_class(self._h, c.ctypes.data_as(C.POINTER(C.c_uint8)))
        return c

    def set_classes(self, c):
        c = np.ascontiguousarray(c, dtype=np.uint8)
        self._lib.om_set_class(self._h, c.ctypes.data_as(C.POINTER(C.c_uint8)))

    def quad_level(self):
        a = np.zeros(self.n, dtype=np.int32)
        self._lib.om_get_quad_level(self._h, a.ctypes.data_as(C.POINTER(C.c_int32)))
        return a

    def set_method_state(self, switched, prev_a=0.0, prev_b=0.0, prev_amax=0.0):
        self._lib.om_set_method_state(self._h, switched, prev_a, prev_b, prev_amax)

    def medial_points(self):
        """(v (n, 4): v1 and v2 of every point, flags (n,) bit 0 / 1: v1 / v2 exist)
        from the triangles of the last rebuild (om_medial_points)."""
        v = np.zeros((self.n, 4))
        f = np.zeros(self.n, dtype=np.uint8)
        self._lib.om_medial_points(self._h, _dp(v), f.ctypes.data_as(C.POINTER(C.c_uint8)))
        return v, f

    def ring(self, i):
        buf = np.zeros(512, dtype=np.int32)
        n = self._lib.om_get_ring(self._h, i, buf.ctypes.data_as(C.POINTER(C.c_int32)), 512)
        return buf[:n].copy()

    def cell_polygon(self, i):
        buf = np.zeros((512, 2))
        n = self._lib.om_get_cell_polygon(self._h, i, _dp(buf), 512)
        return buf[:n].copy()

    def geometry(self):
        nc = self.ncx * self.ncy
        cls = np.zeros(nc, dtype=np.uint8)
        h = np.zeros(nc)
        g = np.zeros(nc)
        havg = np.zeros(1)
        self._lib.om_get_geometry(self._h, cls.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(h), _dp(g), _dp(havg))
        sh = (self.ncy, self.ncx)
        return cls.reshape(sh), h.reshape(sh), g.reshape(sh), float(havg[0])

    def point_cell(self, x, y):
        gi, gj = C.c_int32(), C.c_int32()
        inside = self._lib.om_point_cell(self._h, x, y, C.byref(gi), C.byref(gj))
        return bool(inside), gi.value, gj.value

    def project(self, p_old, old_class, p_new):
        pf = np.zeros(2)
        nc = C.c_int32()
        self._lib.om_project_point(self._h, _dp(_pt(p_old)), old_class, _dp(_pt(p_new)), _dp(pf), C.byref(nc))
        return pf, nc.value
