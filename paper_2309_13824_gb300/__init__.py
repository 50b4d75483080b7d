"""GB300 meshing iteration of TriMe++ (arXiv 2309.13824) behind a C ABI.

This module only marshals arguments to the shared library built from csrc/
(see include/trime.h); every step of the iteration runs in the CUDA kernels.
There is no CPU fallback: importing works without a GPU, but any call needs
the built library and a CUDA device and raises otherwise.

Function names mirror the C ABI.  ``Mesh`` (one mesh) and ``MeshBatch``
(many meshes stepped by the same launches) are small convenience wrappers
that accept numpy arrays and torch tensors and return numpy arrays.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "_build" / "libtrime_gb300.so"

TRIME_OK = 0
TRIME_EINVAL = -1
TRIME_ENOMEM = -2
TRIME_ECUDA = -3
TRIME_ECAPACITY = -4
TRIME_ETIMEOUT = -5
TRIME_EDEVICE = -6


class MeshError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"trime error {code}: {msg}")
        self.code = code


class mesh_grid2d(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("x0", C.c_double), ("y0", C.c_double),
                ("x1", C.c_double), ("y1", C.c_double), ("v", C.POINTER(C.c_float))]


class mesh_params(C.Structure):
    _fields_ = [("precision", C.c_int32), ("method", C.c_int32), ("bounded", C.c_int32),
                ("validity", C.c_int32), ("newton_max", C.c_int32), ("trace_max", C.c_int32),
                ("quad_max_level", C.c_int32), ("debug", C.c_int32), ("fac_F", C.c_double),
                ("k_spring", C.c_double), ("dt", C.c_double), ("fac_pt", C.c_double), ("fac_geps", C.c_double),
                ("fac_voro_bound", C.c_double), ("fac_end", C.c_double), ("T_circ", C.c_double),
                ("T_switch", C.c_double), ("T_end_q", C.c_double), ("T_end_amax", C.c_double),
                ("N_opt", C.c_double), ("eta", C.c_double), ("damping", C.c_double), ("fac_retria", C.c_double),
                ("fac_add", C.c_double), ("T_add", C.c_double), ("n_total", C.c_int64)]


class mesh_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("terminated", C.c_int32), ("method", C.c_int32),
                ("switched", C.c_int32), ("n_tri", C.c_int64), ("n_edges", C.c_int64),
                ("half_mean_alpha", C.c_double), ("half_mean_beta", C.c_double), ("max_alpha", C.c_double),
                ("max_beta", C.c_double), ("min_angle_deg", C.c_double), ("mean_size_dev", C.c_double),
                ("fac_mu", C.c_double), ("exact_calls", C.c_int64), ("clip_inconsistent", C.c_int64),
                ("ring_overflow", C.c_int64), ("exact_overflow", C.c_int64), ("newton_fail", C.c_int64),
                ("trace_cap", C.c_int64), ("quad_cap", C.c_int64), ("dup_points", C.c_int64),
                ("small_moves", C.c_int32), ("target_reached", C.c_int32), ("vor_candidates", C.c_int64),
                ("vor_picks", C.c_int64), ("vor_cuts", C.c_int64), ("vor_rings", C.c_int64), ("vor_wide", C.c_int64),
                ("triangulations", C.c_int64), ("added", C.c_int64), ("n_points", C.c_int64),
                ("vor_fp64", C.c_int64), ("vor_resolve", C.c_int64), ("vor_direct", C.c_int64)]


class mesh_tuning(C.Structure):
    _fields_ = [("n_opt", C.c_double), ("lanes", C.c_int32), ("n_candidates", C.c_int32),
                ("n_slots", C.c_int64), ("n_buckets", C.c_int64), ("cand_n_opt", C.c_double * 12),
                ("cand_lanes", C.c_int32 * 12), ("cand_ms", C.c_double * 12)]


# every symbol include/trime.h declares
EXPORTS = ["mesh_segment_sdf_points", "mesh_adf_build", "mesh_adf_cells", "mesh_adf_size", "mesh_adf_export",
           "mesh_adf_eval", "mesh_adf_destroy", "mesh_default_params", "mesh_init", "mesh_rebuild", "mesh_step", "mesh_get_count", "mesh_get_state", "mesh_segment_sdf_grid", "mesh_sizing_field", "mesh_medial_points", "mesh_auto_sizing", "mesh_init_points", "mesh_get_triangles",
           "mesh_get_points", "mesh_set_state", "mesh_set_method_state", "mesh_get_debug", "mesh_destroy",
           "mesh_last_error", "mesh_bucket_points", "mesh_exact_predicates", "mesh_profile_step",
           "mesh_bucket_points_noalloc", "mesh_batch_init", "mesh_batch_size", "mesh_batch_rebuild",
           "mesh_batch_step", "mesh_batch_get_triangles", "mesh_batch_get_points", "mesh_batch_set_state",
           "mesh_batch_set_method_state", "mesh_batch_profile_step", "mesh_batch_get_tuning", "mesh_batch_destroy",
           "mesh_set_tuning", "mesh_batch_set_tuning", "mesh_tc_gemm_bf16", "mlp_create", "mlp_destroy",
           "mlp_get_params", "mlp_set_params", "mlp_forward", "mlp_loss_grad", "mlp_train", "mesh_features",
           "mesh_collect_pairs", "mesh_propose", "mesh_step_learned", "mesh_set_quality_target",
           "mesh_batch_set_quality_target", "mesh_measure_pipe_peaks", "mesh_batch_step_learned", "mesh_quality",
           "mesh_batch_quality"]

MLP_IN = 48
MLP_PARAMS = 7426

_lib = None


def build(**kw) -> Path:
    from . import buildlib as _b

    return _b.build(**kw)


def lib():
    """Load the CUDA library; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"CUDA library missing: {LIB_PATH} (run paper_2309_13824_gb300.build())")
    L = C.CDLL(str(LIB_PATH))
    P = C.POINTER
    vp = C.c_void_p
    L.mesh_default_params.argtypes = [P(mesh_params)]
    L.mesh_default_params.restype = None
    L.mesh_init.argtypes = [P(vp), P(mesh_grid2d), P(mesh_grid2d), vp, C.c_int64, P(mesh_params), vp]
    L.mesh_rebuild.argtypes = [vp, P(mesh_stats)]
    L.mesh_step.argtypes = [vp, C.c_int32, P(mesh_stats)]
    L.mesh_get_triangles.argtypes = [vp, vp, C.c_int64, P(C.c_int64)]
    L.mesh_get_points.argtypes = [vp, vp, C.c_int64, P(C.c_int64)]
    L.mesh_set_state.argtypes = [vp, vp, vp, vp]
    L.mesh_set_method_state.argtypes = [vp, C.c_int32, C.c_double, C.c_double, C.c_double]
    L.mesh_get_debug.argtypes = [vp, C.c_int32, vp, C.c_int64]
    L.mesh_destroy.argtypes = [vp]
    L.mesh_destroy.restype = None
    L.mesh_last_error.restype = C.c_char_p
    L.mesh_bucket_points.argtypes = [vp, vp, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double,
                                     C.c_int32, C.c_int32, vp, vp, vp, vp]
    L.mesh_exact_predicates.argtypes = [vp, vp, C.c_int64, vp, vp]
    L.mesh_profile_step.argtypes = [vp, C.c_int32, vp]
    L.mesh_bucket_points_noalloc.argtypes = [vp, vp, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double,
                                             C.c_int32, C.c_int32, vp, vp, vp]
    L.mesh_batch_init.argtypes = [P(vp), C.c_int32, P(mesh_grid2d), P(mesh_grid2d), P(vp), P(C.c_int64),
                                  P(mesh_params), C.c_int32, vp]
    L.mesh_batch_size.argtypes = [vp]
    L.mesh_batch_rebuild.argtypes = [vp, vp]
    L.mesh_batch_step.argtypes = [vp, C.c_int32, vp]
    L.mesh_batch_get_triangles.argtypes = [vp, C.c_int32, vp, C.c_int64, P(C.c_int64)]
    L.mesh_batch_get_points.argtypes = [vp, C.c_int32, vp, C.c_int64, P(C.c_int64)]
    L.mesh_batch_set_state.argtypes = [vp, C.c_int32, vp, vp, vp]
    L.mesh_batch_set_method_state.argtypes = [vp, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double]
    L.mesh_batch_profile_step.argtypes = [vp, C.c_int32, vp]
    L.mesh_batch_get_tuning.argtypes = [vp, P(mesh_tuning)]
    L.mesh_set_tuning.argtypes = [vp, C.c_double, C.c_int32]
    L.mesh_tc_gemm_bf16.argtypes = [vp, vp, vp, C.c_int32, C.c_int32, C.c_int32]
    L.mlp_create.argtypes = [P(vp), vp, C.c_uint64, vp]
    L.mlp_destroy.argtypes = [vp]
    L.mlp_destroy.restype = None
    L.mlp_get_params.argtypes = [vp, vp]
    L.mlp_set_params.argtypes = [vp, vp]
    L.mlp_forward.argtypes = [vp, vp, C.c_int64, vp]
    L.mlp_loss_grad.argtypes = [vp, vp, vp, C.c_int64, P(C.c_double), vp]
    L.mlp_train.argtypes = [vp, vp, vp, C.c_int64, C.c_int32, C.c_int32, C.c_double, C.c_uint64, P(C.c_double)]
    L.mesh_features.argtypes = [vp, vp, vp]
    L.mesh_set_quality_target.argtypes = [vp, C.c_double]
    L.mesh_measure_pipe_peaks.argtypes = [P(C.c_double), P(C.c_double), P(C.c_int32), P(C.c_int32)]
    L.mesh_batch_set_quality_target.argtypes = [vp, C.c_int32, C.c_double]
    L.mesh_collect_pairs.argtypes = [vp, C.c_int32, vp, vp]
    L.mesh_propose.argtypes = [vp, vp, C.c_double]
    L.mesh_step_learned.argtypes = [vp, vp, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_int32,
                                    P(mesh_stats), P(C.c_int32), P(C.c_int32)]
    L.mesh_batch_step_learned.argtypes = [vp, vp, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_int32,
                                          P(mesh_stats), P(C.c_int32), P(C.c_int32)]
    L.mesh_batch_set_tuning.argtypes = [vp, C.c_double, C.c_int32]
    L.mesh_quality.argtypes = [vp, P(mesh_quality_stats)]
    L.mesh_batch_quality.argtypes = [vp, C.c_int32, P(mesh_quality_stats)]
    L.mesh_batch_destroy.argtypes = [vp]
    L.mesh_batch_destroy.restype = None
    L.mesh_get_count.argtypes = [vp, P(C.c_int64), P(C.c_int64)]
    L.mesh_get_state.argtypes = [vp, vp, vp, vp]
    L.mesh_segment_sdf_grid.argtypes = [P(C.c_double), C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double,
                                        C.c_int32, C.c_int32, vp, vp]
    L.mesh_sizing_field.argtypes = [P(C.c_double), P(C.c_double), C.c_int64, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_double, C.c_int32, C.c_int32, vp, vp]
    L.mesh_medial_points.argtypes = [vp, P(C.c_double), P(C.c_uint8)]
    L.mesh_auto_sizing.argtypes = [P(C.c_double), C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_int32, C.c_int32, vp, vp, P(C.c_int64), vp]
    L.mesh_init_points.argtypes = [P(mesh_grid2d), P(mesh_grid2d), C.c_int64, C.c_uint64, P(mesh_params),
                                   P(C.c_double), C.c_int64, P(C.c_int64), vp]
    L.mesh_segment_sdf_points.argtypes = [P(C.c_double), C.c_int64, vp, C.c_int64, vp, vp]
    L.mesh_adf_build.argtypes = [P(C.c_double), C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32,
                                 C.c_int32, P(C.c_int32), P(C.c_double), C.c_int32, C.c_int32, P(vp), vp]
    L.mesh_adf_cells.argtypes = [vp, C.c_double, P(C.c_int32), P(C.c_double), C.c_int64, P(C.c_int64)]
    L.mesh_adf_size.argtypes = [vp, P(C.c_int64), P(C.c_int32)]
    L.mesh_adf_export.argtypes = [vp, P(C.c_double), P(C.c_int32), P(C.c_int32), P(C.c_int32), C.c_int64,
                                  P(C.c_int64)]
    L.mesh_adf_eval.argtypes = [vp, vp, C.c_int64, vp, vp]
    L.mesh_adf_destroy.argtypes = [vp]
    L.mesh_adf_destroy.restype = None
    for name in ("mesh_init", "mesh_rebuild", "mesh_step", "mesh_get_count", "mesh_get_state",
                 "mesh_segment_sdf_grid", "mesh_sizing_field", "mesh_medial_points", "mesh_auto_sizing",
                 "mesh_init_points", "mesh_get_triangles", "mesh_get_points",
                 "mesh_set_state", "mesh_set_method_state", "mesh_get_debug", "mesh_bucket_points",
                 "mesh_exact_predicates", "mesh_profile_step", "mesh_bucket_points_noalloc", "mesh_batch_init",
                 "mesh_batch_size", "mesh_batch_rebuild", "mesh_batch_step", "mesh_batch_get_triangles",
                 "mesh_batch_get_points", "mesh_batch_set_state", "mesh_batch_set_method_state",
                 "mesh_batch_profile_step", "mesh_batch_get_tuning", "mesh_set_tuning", "mesh_batch_set_tuning",
                 "mesh_tc_gemm_bf16", "mlp_create", "mlp_get_params", "mlp_set_params", "mlp_forward",
                 "mlp_loss_grad", "mlp_train", "mesh_features", "mesh_collect_pairs", "mesh_propose",
                 "mesh_step_learned", "mesh_set_quality_target", "mesh_batch_set_quality_target",
                 "mesh_measure_pipe_peaks", "mesh_batch_step_learned", "mesh_quality", "mesh_batch_quality", "mesh_segment_sdf_points", "mesh_adf_build", "mesh_adf_cells",
                 "mesh_adf_size", "mesh_adf_export", "mesh_adf_eval"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(rc):
    if rc != TRIME_OK:
        raise MeshError(rc, lib().mesh_last_error().decode())
    return rc


def mesh_default_params() -> mesh_params:
    p = mesh_params()
    lib().mesh_default_params(C.byref(p))
    return p


def mesh_last_error() -> str:
    return lib().mesh_last_error().decode()


def _grid(g):
    v = np.ascontiguousarray(g.values, dtype=np.float32)
    return mesh_grid2d(v.shape[1], v.shape[0], g.x0, g.y0, g.x1, g.y1, v.ctypes.data_as(C.POINTER(C.c_float))), v


def _ptr(t):
    """Raw pointer of a numpy array or torch tensor (device or host)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(t.ctypes.data)


def mesh_bucket_points(x, y, n, box, nbx, nby, bucket_start, sorted_idx, scratch, stream=0):
    """a1 on device arrays (torch CUDA tensors); asynchronous on `stream`."""
    rc = lib().mesh_bucket_points(_ptr(x), _ptr(y), n, box[0], box[1], box[2], box[3], nbx, nby,
                                  _ptr(bucket_start), _ptr(sorted_idx), _ptr(scratch), C.c_void_p(stream))
    return _check(rc)


def mesh_bucket_points_noalloc(x, y, n, box, nbx, nby, bucket_start, sorted_idx, stream=0):
    """mesh_bucket_points without any device allocation (library-owned scratch)."""
    rc = lib().mesh_bucket_points_noalloc(_ptr(x), _ptr(y), n, box[0], box[1], box[2], box[3], nbx, nby,
                                          _ptr(bucket_start), _ptr(sorted_idx), C.c_void_p(stream))
    return _check(rc)


def mesh_exact_predicates(pts, ids):
    """Device exact predicates on (nq, 4, 2) points and (nq, 4) ids."""
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 8)
    ids = np.ascontiguousarray(ids, dtype=np.int32).reshape(-1, 4)
    nq = len(pts)
    o = np.zeros(nq, dtype=np.int32)
    c = np.zeros(nq, dtype=np.int32)
    _check(lib().mesh_exact_predicates(pts.ctypes.data_as(C.c_void_p), ids.ctypes.data_as(C.c_void_p), nq,
                                       o.ctypes.data_as(C.c_void_p), c.ctypes.data_as(C.c_void_p)))
    return o, c


def bf16_bits(x) -> np.ndarray:
    """float32 values rounded to the nearest BF16 (ties to even), as uint16 bits."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = ((u >> 16) & 1) + 0x7FFF
    return ((u + r) >> 16).astype(np.uint16)


def bf16_to_float(b) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def mesh_tc_gemm_bf16(A, B):
    """D = A B^T on the tensor cores (A: M x K, B: N x K BF16 bit arrays)."""
    A = np.ascontiguousarray(A, dtype=np.uint16)
    B = np.ascontiguousarray(B, dtype=np.uint16)
    M, K = A.shape
    N = B.shape[0]
    D = np.zeros((M, N), dtype=np.float32)
    _check(lib().mesh_tc_gemm_bf16(A.ctypes.data_as(C.c_void_p), B.ctypes.data_as(C.c_void_p),
                                   D.ctypes.data_as(C.c_void_p), M, N, K))
    return D


def mesh_measure_pipe_peaks() -> dict:
    """Measured FP32 / FP64 fused-multiply-add throughput of the current device."""
    f32, f64 = C.c_double(), C.c_double()
    sm, clk = C.c_int32(), C.c_int32()
    _check(lib().mesh_measure_pipe_peaks(C.byref(f32), C.byref(f64), C.byref(sm), C.byref(clk)))
    return {"fp32_tflops": f32.value, "fp64_tflops": f64.value, "sm_count": sm.value, "sm_clock_mhz": clk.value / 1e3}


def segment_sdf_grid(verts_cw, n: int, box=(-1.1, -1.1, 1.1, 1.1), ny: int = None, out=None, stream=None):
    """Sec. 3.1 SDF of the clockwise loop verts_cw (k, 2) on an n x ny node
    grid over box (x0, y0, x1, y1) (mesh_segment_sdf_grid): a float32 numpy
    array (ny, n), or written into `out` (host array or device tensor)."""
    v = np.ascontiguousarray(verts_cw, dtype=np.float64).reshape(-1, 2)
    ny = n if ny is None else ny
    x0, y0, x1, y1 = box
    res = out if out is not None else np.empty((ny, n), dtype=np.float32)
    st = C.c_void_p(0 if stream is None else int(stream))
    _check(lib().mesh_segment_sdf_grid(v.ctypes.data_as(C.POINTER(C.c_double)), len(v), x0, y0, x1, y1, n, ny,
                                       _ptr(res), st))
    return res


def sizing_field(samples, lfs, K: float, n: int, box=(-1.1, -1.1, 1.1, 1.1), ny: int = None, out=None,
                 stream=None):
    """Eq. 7 sizing field of boundary samples (k, 2) with local feature sizes
    lfs (k,) and gradation K on an n x ny node grid over box
    (mesh_sizing_field): a float32 numpy array (ny, n), or written into `out`."""
    s = np.ascontiguousarray(samples, dtype=np.float64).reshape(-1, 2)
    lf = np.ascontiguousarray(lfs, dtype=np.float64).ravel()
    ny = n if ny is None else ny
    x0, y0, x1, y1 = box
    res = out if out is not None else np.empty((ny, n), dtype=np.float32)
    st = C.c_void_p(0 if stream is None else int(stream))
    _check(lib().mesh_sizing_field(s.ctypes.data_as(C.POINTER(C.c_double)), lf.ctypes.data_as(C.POINTER(C.c_double)),
                                   len(s), float(K), x0, y0, x1, y1, n, ny, _ptr(res), st))
    return res


def segment_sdf_points(verts_cw, pts, out=None, stream=None):
    """Exact FP64 signed distance of the clockwise loop verts_cw at the
    points pts (n, 2) (mesh_segment_sdf_points): a numpy array, or written
    into `out` (numpy or CUDA tensor of n float64)."""
    v = np.ascontiguousarray(verts_cw, dtype=np.float64).reshape(-1, 2)
    if not hasattr(pts, "data_ptr"):
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    n = pts.shape[0]
    res = out if out is not None else np.empty(n)
    st = C.c_void_p(0 if stream is None else int(stream))
    _check(lib().mesh_segment_sdf_points(v.ctypes.data_as(C.POINTER(C.c_double)), len(v), _ptr(pts), n, _ptr(res),
                                         st))
    return res


class ADF:
    """Adaptive distance field of a clockwise polygon (Sec. 3.7; a handle to
    adf_t): one quadtree per listed grid cell, refined until the bilinear
    error at the edge midpoints and centre is within the cell's tolerance."""

    def __init__(self, verts_cw, box, nx: int, ny: int, cells, tol, max_depth: int = 10, stream=None):
        self._v = np.ascontiguousarray(verts_cw, dtype=np.float64).reshape(-1, 2)
        c = np.ascontiguousarray(cells, dtype=np.int32).ravel()
        t = np.ascontiguousarray(tol, dtype=np.float64).ravel()
        self.box, self.nx, self.ny = tuple(float(b) for b in box), int(nx), int(ny)
        self.cells = c.copy()
        h = C.c_void_p()
        st = C.c_void_p(0 if stream is None else int(stream))
        x0, y0, x1, y1 = self.box
        _check(lib().mesh_adf_build(self._v.ctypes.data_as(C.POINTER(C.c_double)), len(self._v), x0, y0, x1, y1,
                                    self.nx, self.ny, c.ctypes.data_as(C.POINTER(C.c_int32)),
                                    t.ctypes.data_as(C.POINTER(C.c_double)), len(c), int(max_depth), C.byref(h), st))
        self._h = h

    @classmethod
    def for_mesh(cls, mesh, verts_cw, sdf_grid, fac_etol: float = 0.1, max_depth: int = 10, stream=None):
        """The paper's ADF of a mesh: its boundary cells and tolerances
        (mesh_adf_cells) on its SDF grid `sdf_grid` (the Grid it was made with)."""
        n = C.c_int64()
        L = lib()
        rc = L.mesh_adf_cells(mesh._h, float(fac_etol), None, None, 0, C.byref(n))
        if rc not in (0, -4):
            _check(rc)
        cells = np.zeros(n.value, np.int32)
        tol = np.zeros(n.value)
        _check(L.mesh_adf_cells(mesh._h, float(fac_etol), cells.ctypes.data_as(C.POINTER(C.c_int32)),
                                tol.ctypes.data_as(C.POINTER(C.c_double)), len(cells), C.byref(n)))
        g = sdf_grid
        obj = cls(verts_cw, (g.x0, g.y0, g.x1, g.y1), g.values.shape[1], g.values.shape[0], cells, tol, max_depth,
                  stream)
        obj.tol = tol
        return obj

    def size(self):
        n, lv = C.c_int64(), C.c_int32()
        _check(lib().mesh_adf_size(self._h, C.byref(n), C.byref(lv)))
        return n.value, lv.value

    def nodes(self):
        """(v (n, 4), child (n,), root (n,), lev (n, 3)) in build order."""
        n = self.size()[0]
        v = np.zeros((n, 4))
        child = np.zeros(n, np.int32)
        root = np.zeros(n, np.int32)
        lev = np.zeros((n, 3), np.int32)
        got = C.c_int64()
        ip = C.POINTER(C.c_int32)
        _check(lib().mesh_adf_export(self._h, v.ctypes.data_as(C.POINTER(C.c_double)), child.ctypes.data_as(ip),
                                     root.ctypes.data_as(ip), lev.ctypes.data_as(ip), n, C.byref(got)))
        return v, child, root, lev

    def eval(self, pts, out=None, stream=None):
        """ADF values at pts (n, 2) (numpy or CUDA tensor); NaN outside the trees."""
        if not hasattr(pts, "data_ptr"):
            pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
        n = pts.shape[0]
        res = out if out is not None else np.empty(n)
        st = C.c_void_p(0 if stream is None else int(stream))
        _check(lib().mesh_adf_eval(self._h, _ptr(pts), n, _ptr(res), st))
        return res

    def close(self):
        if getattr(self, "_h", None):
            lib().mesh_adf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def auto_sizing(verts_cw, K: float, n: int, box=(-1.1, -1.1, 1.1, 1.1), ny: int = None, stream=None):
    """The automatic sizing pipeline (App. A, Sec. 3.3, Eq. 7; mesh_auto_sizing)
    for a clockwise polygon on an n x ny node grid: (SDF grid, sizing grid) as
    float32 numpy arrays (ny, n) and the counts {samples, medial, kept}."""
    v = np.ascontiguousarray(verts_cw, dtype=np.float64).reshape(-1, 2)
    ny = n if ny is None else ny
    x0, y0, x1, y1 = box
    sdf = np.empty((ny, n), dtype=np.float32)
    mu = np.empty((ny, n), dtype=np.float32)
    cnt = (C.c_int64 * 3)()
    st = C.c_void_p(0 if stream is None else int(stream))
    _check(lib().mesh_auto_sizing(v.ctypes.data_as(C.POINTER(C.c_double)), len(v), float(K), x0, y0, x1, y1, n, ny,
                                  _ptr(sdf), _ptr(mu), cnt, st))
    return sdf, mu, {"samples": cnt[0], "medial": cnt[1], "kept": cnt[2]}


def init_points(sdf, sizing, n_init: int, seed: int = 0, stream=None, **params) -> np.ndarray:
    """Sec. 3.5 initial points (mesh_init_points): (n, 2) float64."""
    p = _params(params)
    gs, ks = _grid(sdf)
    gz, kz = _grid(sizing)
    n = C.c_int64()
    st = C.c_void_p(0 if stream is None else int(stream))
    rc = lib().mesh_init_points(C.byref(gs), C.byref(gz), int(n_init), int(seed), C.byref(p), None, 0, C.byref(n), st)
    if rc not in (TRIME_OK, TRIME_ECAPACITY):
        _check(rc)
    out = np.empty((n.value, 2))
    _check(lib().mesh_init_points(C.byref(gs), C.byref(gz), int(n_init), int(seed), C.byref(p),
                                  out.ctypes.data_as(C.POINTER(C.c_double)), n.value, C.byref(n), st))
    return out


def _stats_dict(s: mesh_stats) -> dict:
    return {name: getattr(s, name) for name, _ in mesh_stats._fields_}


class mesh_quality_stats(C.Structure):
    _fields_ = [("n_tri", C.c_int64), ("n_edges", C.c_int64), ("median_alpha", C.c_double),
                ("median_beta", C.c_double), ("mean_alpha", C.c_double), ("mean_beta", C.c_double),
                ("max_alpha", C.c_double), ("max_beta", C.c_double), ("std_alpha", C.c_double),
                ("std_beta", C.c_double), ("frac_alpha_lt_1_2", C.c_double), ("frac_alpha_lt_2", C.c_double),
                ("min_angle_deg", C.c_double), ("alpha_hist", C.c_int64 * 10), ("fac_mu", C.c_double),
                ("mean_size_dev", C.c_double), ("p95_size_dev", C.c_double)]


ALPHA_BIN_EDGES = (1.0, 1.05, 1.1, 1.2, 1.3, 1.5, 2.0, 3.0, 5.0, 10.0)


def _quality_dict(q: mesh_quality_stats) -> dict:
    d = {name: getattr(q, name) for name, _ in mesh_quality_stats._fields_}
    d["alpha_hist"] = list(q.alpha_hist)
    return d


class Mesh:
    """One mesh on the current CUDA device (a handle to mesh_t)."""

    def __init__(self, sdf, sizing, xy, stream=None, **params):
        L = lib()
        p = _params(params)
        self.params = p
        self.precision = p.precision
        self.dtype = np.float64 if p.precision == 0 else np.float32
        xy = np.ascontiguousarray(np.asarray(xy, dtype=self.dtype).reshape(-1, 2))
        gs, ks = _grid(sdf)
        gz, kz = _grid(sizing)
        h = C.c_void_p()
        st = C.c_void_p(0 if stream is None else int(stream))
        rc = L.mesh_init(C.byref(h), C.byref(gs), C.byref(gz), xy.ctypes.data_as(C.c_void_p), len(xy),
                         C.byref(p), st)
        _check(rc)
        self._h = h

    @property
    def n(self) -> int:
        """N_current: the number of points (grows under point addition)."""
        c = C.c_int64()
        _check(lib().mesh_get_count(self._h, C.byref(c), None))
        return c.value

    @property
    def n_total(self) -> int:
        c = C.c_int64()
        _check(lib().mesh_get_count(self._h, None, C.byref(c)))
        return c.value

    def close(self):
        if getattr(self, "_h", None):
            lib().mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rebuild(self) -> dict:
        s = mesh_stats()
        _check(lib().mesh_rebuild(self._h, C.byref(s)))
        return _stats_dict(s)

    def step(self, n_iters: int = 1, check=True) -> dict:
        s = mesh_stats()
        rc = lib().mesh_step(self._h, n_iters, C.byref(s))
        if check:
            _check(rc)
        d = _stats_dict(s)
        d["rc"] = rc
        return d

    def step_async(self, n_iters: int = 1):
        """Enqueue iterations on the mesh's stream without reading back."""
        _check(lib().mesh_step(self._h, n_iters, None))

    def profile(self, n_iters: int = 1):
        """Per-stage device milliseconds summed over n_iters iterations."""
        ms = np.zeros(7)
        _check(lib().mesh_profile_step(self._h, n_iters, ms.ctypes.data_as(C.c_void_p)))
        return dict(zip(["bucket", "voronoi", "emit", "stats", "update", "post", "total"], ms))

    def quality(self) -> dict:
        """mesh_quality: the quality report of the last rebuild."""
        q = mesh_quality_stats()
        _check(lib().mesh_quality(self._h, C.byref(q)))
        return _quality_dict(q)

    def triangles(self, out=None):
        """Valid triangles (int32, smallest id first, CCW), order unspecified.
        With `out` (host array or device tensor of shape (cap, 3)) fills it
        and returns the count; otherwise returns a numpy array."""
        L = lib()
        n = C.c_int64()
        if out is not None:
            _check(L.mesh_get_triangles(self._h, _ptr(out), out.shape[0], C.byref(n)))
            return n.value
        rc = L.mesh_get_triangles(self._h, None, 0, C.byref(n))
        if rc not in (TRIME_OK, TRIME_ECAPACITY):
            _check(rc)
        t = np.zeros((n.value, 3), dtype=np.int32)
        if n.value:
            _check(L.mesh_get_triangles(self._h, t.ctypes.data_as(C.c_void_p), n.value, C.byref(n)))
        return t

    def points(self, out=None):
        n = C.c_int64()
        if out is not None:
            _check(lib().mesh_get_points(self._h, _ptr(out), out.shape[0], C.byref(n)))
            return out
        p = np.zeros((self.n, 2), dtype=self.dtype)
        _check(lib().mesh_get_points(self._h, p.ctypes.data_as(C.c_void_p), self.n, C.byref(n)))
        return p

    def set_state(self, xy=None, cls=None, dprev=None):
        a = None if xy is None else np.ascontiguousarray(np.asarray(xy, dtype=self.dtype).reshape(-1, 2))
        b = None if cls is None else np.ascontiguousarray(cls, dtype=np.uint8)
        c = None if dprev is None else np.ascontiguousarray(dprev, dtype=np.float64)
        _check(lib().mesh_set_state(self._h, None if a is None else a.ctypes.data_as(C.c_void_p),
                                    None if b is None else b.ctypes.data_as(C.c_void_p),
                                    None if c is None else c.ctypes.data_as(C.c_void_p)))

    def set_method_state(self, switched, prev_a=0.0, prev_b=0.0, prev_amax=0.0):
        _check(lib().mesh_set_method_state(self._h, switched, prev_a, prev_b, prev_amax))

    def state(self):
        """(positions, classes, previous move distances) in input order."""
        n = self.n
        xy = np.zeros((n, 2), dtype=self.dtype)
        cls = np.zeros(n, dtype=np.uint8)
        dp = np.zeros(n)
        _check(lib().mesh_get_state(self._h, xy.ctypes.data_as(C.c_void_p), cls.ctypes.data_as(C.c_void_p),
                                    dp.ctypes.data_as(C.c_void_p)))
        return xy, cls, dp

    def set_tuning(self, n_opt: float, lanes: int = 8):
        _check(lib().mesh_set_tuning(self._h, n_opt, lanes))

    def medial_points(self):
        """(v (n, 4): v1 and v2 of every point, flags (n,) bit 0 / 1: present), Sec. 3.3."""
        n = self.n
        v = np.zeros((n, 4))
        f = np.zeros(n, dtype=np.uint8)
        _check(lib().mesh_medial_points(self._h, v.ctypes.data_as(C.POINTER(C.c_double)),
                                        f.ctypes.data_as(C.POINTER(C.c_uint8))))
        return v, f

    def set_quality_target(self, min_angle_deg: float):
        _check(lib().mesh_set_quality_target(self._h, min_angle_deg))

    # ---- learned proposals
    def features(self):
        """(n, 48) BF16 feature bits (uint16) and h_i (float32), input order."""
        X = np.zeros((self.n, MLP_IN), dtype=np.uint16)
        h = np.zeros(self.n, dtype=np.float32)
        _check(lib().mesh_features(self._h, X.ctypes.data_as(C.c_void_p), h.ctypes.data_as(C.c_void_p)))
        return X, h

    def collect_pairs(self, horizon: int, X, T):
        """One plain iteration, then the features into X (device (n, 48)
        int16/uint16 tensor) and the displacement / h_i over `horizon` more
        plain iterations into T (device (n, 2) float32)."""
        _check(lib().mesh_collect_pairs(self._h, horizon, _ptr(X), _ptr(T)))

    def propose(self, net: "MLP", jump: float = 4.0):
        _check(lib().mesh_propose(self._h, net._h, jump))

    def step_learned(self, net: "MLP", n_iters: int, every: int = 5, jump: float = 5.0, min_angle_tol: float = 0.5,
                     max_proposals: int = 8):
        s = mesh_stats()
        acc, rej = C.c_int32(), C.c_int32()
        _check(lib().mesh_step_learned(self._h, net._h, n_iters, every, jump, min_angle_tol, max_proposals,
                                       C.byref(s), C.byref(acc), C.byref(rej)))
        d = _stats_dict(s)
        d["accepted"], d["rejected"] = acc.value, rej.value
        return d

    def debug(self, what: int):
        width = [2, 2, 2, 1, 1, 1, 1][what]
        out = np.zeros(width * self.n)
        _check(lib().mesh_get_debug(self._h, what, out.ctypes.data_as(C.c_void_p), len(out)))
        return out.reshape(self.n, 2) if width == 2 else out


def _params(params) -> mesh_params:
    p = mesh_default_params()
    for k, v in params.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class MeshBatch:
    """Several independent meshes stepped by the same launches (a handle to
    mesh_batch_t).  `meshes` is a sequence of (sdf, sizing, xy) triples."""

    def __init__(self, meshes, stream=None, autotune=True, **params):
        L = lib()
        p = _params(params)
        self.params = p
        self.dtype = np.float64 if p.precision == 0 else np.float32
        nm = len(meshes)
        self.size = nm
        G = (mesh_grid2d * nm)()
        Z = (mesh_grid2d * nm)()
        X = (C.c_void_p * nm)()
        N = (C.c_int64 * nm)()
        self._keep = []
        self.ns = []
        for k, (sdf, siz, xy) in enumerate(meshes):
            gs, ks = _grid(sdf)
            gz, kz = _grid(siz)
            xy = np.ascontiguousarray(np.asarray(xy, dtype=self.dtype).reshape(-1, 2))
            G[k] = gs
            Z[k] = gz
            X[k] = xy.ctypes.data_as(C.c_void_p)
            N[k] = len(xy)
            self.ns.append(len(xy))
            self._keep += [ks, kz, xy]
        h = C.c_void_p()
        st = C.c_void_p(0 if stream is None else int(stream))
        rc = L.mesh_batch_init(C.byref(h), nm, G, Z, X, N, C.byref(p), 1 if autotune else 0, st)
        self._keep = None
        _check(rc)
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().mesh_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rebuild(self):
        s = (mesh_stats * self.size)()
        _check(lib().mesh_batch_rebuild(self._h, s))
        return [_stats_dict(x) for x in s]

    def step(self, n_iters: int = 1, check=True):
        s = (mesh_stats * self.size)()
        rc = lib().mesh_batch_step(self._h, n_iters, s)
        if check:
            _check(rc)
        return [_stats_dict(x) for x in s]

    def step_async(self, n_iters: int = 1):
        _check(lib().mesh_batch_step(self._h, n_iters, None))

    def step_learned(self, net: "MLP", n_iters: int, every: int = 5, jump: float = 5.0, min_angle_tol: float = 0.5,
                     max_rounds: int = 8):
        """mesh_batch_step_learned: per-mesh statistics with the proposals
        each mesh kept ("accepted") and undid ("rejected")."""
        s = (mesh_stats * self.size)()
        acc = (C.c_int32 * self.size)()
        rej = (C.c_int32 * self.size)()
        _check(lib().mesh_batch_step_learned(self._h, net._h, n_iters, every, jump, min_angle_tol, max_rounds, s,
                                             acc, rej))
        out = [_stats_dict(x) for x in s]
        for k, d in enumerate(out):
            d["accepted"], d["rejected"] = acc[k], rej[k]
        return out

    def profile(self, n_iters: int = 1):
        ms = np.zeros(7)
        _check(lib().mesh_batch_profile_step(self._h, n_iters, ms.ctypes.data_as(C.c_void_p)))
        return dict(zip(["bucket", "voronoi", "emit", "stats", "update", "post", "total"], ms))

    def set_tuning(self, n_opt: float, lanes: int = 8):
        _check(lib().mesh_batch_set_tuning(self._h, n_opt, lanes))

    def set_quality_target(self, min_angle_deg: float, mesh: int = -1):
        _check(lib().mesh_batch_set_quality_target(self._h, mesh, min_angle_deg))

    def tuning(self) -> dict:
        t = mesh_tuning()
        _check(lib().mesh_batch_get_tuning(self._h, C.byref(t)))
        nc = t.n_candidates
        return {"n_opt": t.n_opt, "lanes": t.lanes, "n_slots": t.n_slots, "n_buckets": t.n_buckets,
                "candidates": [(t.cand_n_opt[k], t.cand_lanes[k], t.cand_ms[k]) for k in range(nc)]}

    def quality(self, mesh: int) -> dict:
        q = mesh_quality_stats()
        _check(lib().mesh_batch_quality(self._h, mesh, C.byref(q)))
        return _quality_dict(q)

    def triangles(self, mesh: int):
        L = lib()
        n = C.c_int64()
        rc = L.mesh_batch_get_triangles(self._h, mesh, None, 0, C.byref(n))
        if rc not in (TRIME_OK, TRIME_ECAPACITY):
            _check(rc)
        t = np.zeros((n.value, 3), dtype=np.int32)
        if n.value:
            _check(L.mesh_batch_get_triangles(self._h, mesh, t.ctypes.data_as(C.c_void_p), n.value, C.byref(n)))
        return t

    def points(self, mesh: int, out=None):
        n = C.c_int64()
        if out is not None:
            _check(lib().mesh_batch_get_points(self._h, mesh, _ptr(out), out.shape[0], C.byref(n)))
            return out
        p = np.zeros((self.ns[mesh], 2), dtype=self.dtype)
        _check(lib().mesh_batch_get_points(self._h, mesh, p.ctypes.data_as(C.c_void_p), self.ns[mesh],
                                           C.byref(n)))
        return p

    def set_state(self, mesh: int, xy=None, cls=None, dprev=None):
        a = None if xy is None else np.ascontiguousarray(np.asarray(xy, dtype=self.dtype).reshape(-1, 2))
        b = None if cls is None else np.ascontiguousarray(cls, dtype=np.uint8)
        c = None if dprev is None else np.ascontiguousarray(dprev, dtype=np.float64)
        _check(lib().mesh_batch_set_state(self._h, mesh, None if a is None else a.ctypes.data_as(C.c_void_p),
                                          None if b is None else b.ctypes.data_as(C.c_void_p),
                                          None if c is None else c.ctypes.data_as(C.c_void_p)))

    def set_method_state(self, mesh: int, switched, prev_a=0.0, prev_b=0.0, prev_amax=0.0):
        _check(lib().mesh_batch_set_method_state(self._h, mesh, switched, prev_a, prev_b, prev_amax))


class MLP:
    """The learned displacement model (a handle to mlp_t)."""

    def __init__(self, params=None, seed: int = 0, stream=None):
        h = C.c_void_p()
        p = None
        if params is not None:
            p = np.ascontiguousarray(params, dtype=np.float32).reshape(MLP_PARAMS)
        st = C.c_void_p(0 if stream is None else int(stream))
        _check(lib().mlp_create(C.byref(h), None if p is None else p.ctypes.data_as(C.c_void_p), seed, st))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        p = np.zeros(MLP_PARAMS, dtype=np.float32)
        _check(lib().mlp_get_params(self._h, p.ctypes.data_as(C.c_void_p)))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32).reshape(MLP_PARAMS)
        _check(lib().mlp_set_params(self._h, p.ctypes.data_as(C.c_void_p)))

    def forward(self, X):
        """Y (n, 2) for BF16 feature bits X (n, 48): numpy arrays, or device tensors (then Y is a device tensor)."""
        if hasattr(X, "data_ptr"):
            import torch

            Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
            _check(lib().mlp_forward(self._h, _ptr(X), X.shape[0], _ptr(Y)))
            return Y
        X = np.ascontiguousarray(X, dtype=np.uint16).reshape(-1, MLP_IN)
        Y = np.zeros((len(X), 2), dtype=np.float32)
        _check(lib().mlp_forward(self._h, X.ctypes.data_as(C.c_void_p), len(X), Y.ctypes.data_as(C.c_void_p)))
        return Y

    def loss_grad(self, X, T):
        X = np.ascontiguousarray(X, dtype=np.uint16).reshape(-1, MLP_IN)
        T = np.ascontiguousarray(T, dtype=np.float32).reshape(-1, 2)
        g = np.zeros(MLP_PARAMS, dtype=np.float32)
        loss = C.c_double()
        _check(lib().mlp_loss_grad(self._h, X.ctypes.data_as(C.c_void_p), T.ctypes.data_as(C.c_void_p), len(X),
                                   C.byref(loss), g.ctypes.data_as(C.c_void_p)))
        return loss.value, g

    def train(self, X, T, epochs: int = 1, batch: int = 8192, lr: float = 1e-3, seed: int = 0) -> float:
        """Adam on device tensors X (n, 48) uint16/int16 and T (n, 2) float32; returns the last epoch's loss."""
        loss = C.c_double()
        _check(lib().mlp_train(self._h, _ptr(X), _ptr(T), X.shape[0], epochs, batch, lr, seed, C.byref(loss)))
        return loss.value
