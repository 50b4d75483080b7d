"""Seeded synthetic inputs for the meshing iteration.

This module is the only code shared by the CUDA path's tests/benchmarks and the
CPU oracle.  It holds no meshing arithmetic: it only builds signed-distance and
sizing grids for analytic shapes and draws seeded point sets.

Shapes follow the paper's input conventions (TriMe++, Sec. 3.1): the SDF is
negative inside, positive outside; set difference of two shapes is
max(sdf_A, -sdf_B).  Grids are node-centred, row-major ``values[j, i]`` at
``(x0 + i*dx, y0 + j*dy)``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BOX = (-1.1, -1.1, 1.1, 1.1)


@dataclass
class Grid:
    """A node-centred bilinear grid over the box (x0, y0)-(x1, y1)."""

    values: np.ndarray  # float32, shape (ny, nx)
    x0: float
    y0: float
    x1: float
    y1: float

    @property
    def nx(self) -> int:
        return int(self.values.shape[1])

    @property
    def ny(self) -> int:
        return int(self.values.shape[0])

    def nodes(self):
        xs = np.linspace(self.x0, self.x1, self.nx)
        ys = np.linspace(self.y0, self.y1, self.ny)
        return np.meshgrid(xs, ys)


def _node_grid(n: int, box=BOX):
    x0, y0, x1, y1 = box
    xs = x0 + np.arange(n) * ((x1 - x0) / (n - 1))
    ys = y0 + np.arange(n) * ((y1 - y0) / (n - 1))
    return np.meshgrid(xs, ys)


def disk_sdf_fn(x, y, r=1.0, cx=0.0, cy=0.0):
    return np.hypot(x - cx, y - cy) - r


def annulus_sdf_fn(x, y, r_in=0.3, r_out=1.0):
    return np.maximum(np.hypot(x, y) - r_out, -(np.hypot(x, y) - r_in))


def square_sdf_fn(x, y, lo=0.0, hi=1.0):
    c = 0.5 * (lo + hi)
    h = 0.5 * (hi - lo)
    dx = np.abs(x - c) - h
    dy = np.abs(y - c) - h
    out = np.hypot(np.maximum(dx, 0), np.maximum(dy, 0))
    return out + np.minimum(np.maximum(dx, dy), 0)


def grid_from_fn(fn, n: int, box=BOX) -> Grid:
    X, Y = _node_grid(n, box)
    return Grid(np.ascontiguousarray(fn(X, Y), dtype=np.float32), *box)


def constant_grid(value: float, n: int = 2, box=BOX) -> Grid:
    return Grid(np.full((n, n), value, dtype=np.float32), *box)


# ---------------------------------------------------------------- star polygons
def star_polygon(nv: int, rmin: float, rmax: float, seed: int):
    """Vertices at angles 2*pi*k/nv with radii U[rmin, rmax], listed clockwise."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(rmin, rmax, nv)
    th = 2 * np.pi * np.arange(nv) / nv
    v = np.stack([r * np.cos(th), r * np.sin(th)], 1)
    return v[::-1].copy()  # clockwise (Sec. 3.1 input convention)


def _star_radius(verts_ccw, theta):
    """Radius of the star-shaped polygon boundary along direction theta."""
    nv = len(verts_ccw)
    ang = np.arctan2(verts_ccw[:, 1], verts_ccw[:, 0]) % (2 * np.pi)
    order = np.argsort(ang)
    v = verts_ccw[order]
    ang = ang[order]
    t = theta % (2 * np.pi)
    k = np.searchsorted(ang, t, side="right") - 1
    a = v[k % nv]
    b = v[(k + 1) % nv]
    d = np.stack([np.cos(t), np.sin(t)], -1)
    e = b - a
    # solve s*d = a + u*e
    den = d[..., 0] * e[..., 1] - d[..., 1] * e[..., 0]
    s = (a[..., 0] * e[..., 1] - a[..., 1] * e[..., 0]) / den
    return s


def polygon_sdf_grid(verts_cw, n: int, box=BOX) -> Grid:
    """Signed distance to a star polygon: nearest-segment distance, sign from
    the radial inside test (the polygon is star-shaped around the origin)."""
    from scipy.spatial import cKDTree

    X, Y = _node_grid(n, box)
    P = np.stack([X.ravel(), Y.ravel()], 1)
    a = verts_cw
    b = np.roll(verts_cw, -1, axis=0)
    h = (box[2] - box[0]) / (n - 1)
    seg_len = np.hypot(*(b - a).T)
    k_per = np.maximum(2, np.ceil(seg_len / (h / 4)).astype(int))
    samples, owner = [], []
    for s in range(len(a)):
        t = np.linspace(0, 1, k_per[s], endpoint=False)
        samples.append(a[s] + t[:, None] * (b[s] - a[s]))
        owner.append(np.full(k_per[s], s))
    samples = np.concatenate(samples)
    owner = np.concatenate(owner)
    tree = cKDTree(samples)
    best = np.full(len(P), np.inf)
    _, idx = tree.query(P, k=1)
    nseg = len(a)
    for off in (-1, 0, 1):
        s = (owner[idx] + off) % nseg
        A, B = a[s], b[s]
        e = B - A
        tt = np.clip(((P - A) * e).sum(1) / (e * e).sum(1), 0, 1)
        d = np.hypot(*(P - (A + tt[:, None] * e)).T)
        best = np.minimum(best, d)
    ccw = verts_cw[::-1]
    rr = _star_radius(ccw, np.arctan2(P[:, 1], P[:, 0]))
    inside = np.hypot(P[:, 0], P[:, 1]) < rr
    sdf = np.where(inside, -best, best).reshape(X.shape)
    return Grid(np.ascontiguousarray(sdf, dtype=np.float32), *box)


# ---------------------------------------------------------------- point seeding
def uniform_in(sdf_fn, n: int, seed: int, box=BOX, margin: float = 0.0):
    """n points uniform in {sdf_fn < -margin} by rejection, numpy PCG64."""
    rng = np.random.default_rng(seed)
    out = []
    got = 0
    x0, y0, x1, y1 = box
    while got < n:
        m = max(1024, 2 * (n - got))
        p = np.stack([rng.uniform(x0, x1, m), rng.uniform(y0, y1, m)], 1)
        p = p[sdf_fn(p[:, 0], p[:, 1]) < -margin]
        out.append(p)
        got += len(p)
    return np.ascontiguousarray(np.concatenate(out)[:n], dtype=np.float64)


def density_in(sdf_fn, h_fn, n: int, seed: int, box=BOX, margin: float = 0.0):
    """n points in {sdf_fn < -margin} with density proportional to 1/h^2."""
    rng = np.random.default_rng(seed)
    X, Y = _node_grid(257, box)
    hmin = float(np.min(h_fn(X, Y)))
    out = []
    got = 0
    x0, y0, x1, y1 = box
    while got < n:
        m = max(4096, 4 * (n - got))
        p = np.stack([rng.uniform(x0, x1, m), rng.uniform(y0, y1, m)], 1)
        p = p[sdf_fn(p[:, 0], p[:, 1]) < -margin]
        acc = rng.uniform(0, 1, len(p)) < (hmin / h_fn(p[:, 0], p[:, 1])) ** 2
        p = p[acc]
        out.append(p)
        got += len(p)
    return np.ascontiguousarray(np.concatenate(out)[:n], dtype=np.float64)


# ---------------------------------------------------------------- named workloads
@dataclass
class Workload:
    name: str
    sdf: Grid
    sizing: Grid
    points: np.ndarray  # (N, 2) float64
    method: int  # 0 DM, 1 CVD, 2 hybrid
    precision: int  # 0 FP64, 1 FP32 positions
    iters: int


def disk_workload(n: int = 10_000, seed: int = 0, sdf_n: int = 256, h: float = 0.01) -> Workload:
    """Unit disk, analytic SDF on a sdf_n^2 grid, uniform sizing, uniform seeding."""
    sdf = grid_from_fn(disk_sdf_fn, sdf_n)
    siz = constant_grid(h, 256)
    pts = uniform_in(disk_sdf_fn, n, seed)
    return Workload(f"disk-dm-fp64-n{n}", sdf, siz, pts, 0, 0, 50)


def annulus_h_fn(x, y):
    return 0.002 + 0.05 * np.abs(annulus_sdf_fn(x, y))


def annulus_workload(n: int = 1_000_000, seed: int = 1, sdf_n: int = 1024, siz_n: int = 512,
                     method: int = 2, precision: int = 0) -> Workload:
    """Annulus 0.3 <= r <= 1, adaptive sizing 0.002 + 0.05|sdf|, density 1/h^2."""
    sdf = grid_from_fn(annulus_sdf_fn, sdf_n)
    siz = grid_from_fn(annulus_h_fn, siz_n)
    pts = density_in(annulus_sdf_fn, annulus_h_fn, n, seed)
    mname = {0: "dm", 1: "cvd", 2: "hybrid"}[method]
    pname = {0: "fp64", 1: "fp32"}[precision]
    return Workload(f"annulus-{mname}-{pname}-n{n}", sdf, siz, pts, method, precision, 200)


def square_workload(n: int, seed: int = 4, sdf_n: int = 256) -> Workload:
    """Paper-shaped uniform square [0,1]^2 inside the [-1.1,1.1]^2 box."""
    sdf = grid_from_fn(square_sdf_fn, sdf_n)
    siz = constant_grid(1.0, 2)
    pts = uniform_in(square_sdf_fn, n, seed)
    return Workload(f"square-n{n}", sdf, siz, pts, 2, 0, 100)


def star_workload(n: int, nv: int = 500, seed: int = 2, sdf_n: int = 1024, siz_n: int = 256,
                  precision: int = 1) -> Workload:
    """Random star polygon; sizing clamp(0.1*dist_to_boundary + 0.01*r_local, 2e-4, 1e-2)."""
    verts = star_polygon(nv, 0.4, 1.0, seed)
    sdf = polygon_sdf_grid(verts, sdf_n)
    coarse = polygon_sdf_grid(verts, siz_n)
    # local thickness proxy: each vertex's distance to the nearest non-incident vertex
    from scipy.spatial import cKDTree

    tree = cKDTree(verts)
    dd, _ = tree.query(verts, k=3)
    lfs = dd[:, 2]
    Xs, Ys = coarse.nodes()
    _, vi = tree.query(np.stack([Xs.ravel(), Ys.ravel()], 1), k=1)
    h = np.clip(0.1 * np.abs(coarse.values.ravel()) + 0.25 * lfs[vi], 2e-4, 1e-2)
    siz = Grid(np.ascontiguousarray(h.reshape(coarse.values.shape), dtype=np.float32),
               coarse.x0, coarse.y0, coarse.x1, coarse.y1)

    def sdf_fn(x, y):
        return _bilinear_np(sdf, x, y)

    def h_fn(x, y):
        return _bilinear_np(siz, x, y)

    pts = density_in(sdf_fn, h_fn, n, seed + 1, margin=0.0)
    return Workload(f"star{nv}-hybrid-n{n}", sdf, siz, pts, 2, precision, 100)


@dataclass
class BatchWorkload:
    name: str
    meshes: list  # (sdf Grid, sizing Grid, points (N, 2) float64) per mesh
    method: int
    precision: int
    iters: int

    @property
    def total_points(self) -> int:
        return int(sum(len(m[2]) for m in self.meshes))


def _star_batch_member(args):
    nv, n, vseed, pseed, sdf_n = args
    verts = star_polygon(nv, 0.4, 1.0, vseed)
    sdf = polygon_sdf_grid(verts, sdf_n)
    siz = Grid(np.ascontiguousarray(0.002 + 0.05 * np.abs(sdf.values), dtype=np.float32),
               sdf.x0, sdf.y0, sdf.x1, sdf.y1)

    def sdf_fn(x, y):
        return _bilinear_np(sdf, x, y)

    return sdf, siz, uniform_in(sdf_fn, n, pseed)


def star_batch_workload(n_meshes: int = 256, seed: int = 7, sdf_n: int = 512, n_min: float = 1e3,
                        n_max: float = 1e5, nv_min: int = 50, nv_max: int = 300, precision: int = 1,
                        workers: int = 0) -> BatchWorkload:
    """Independent random star polygons (nv_min..nv_max vertices, radii
    U[0.4, 1]), SDF on sdf_n^2, sizing 0.002 + 0.05|sdf| on the same nodes,
    point counts log-uniform in [n_min, n_max], uniform seeding inside each
    shape.  workers > 1 builds the meshes in that many spawned processes."""
    rng = np.random.default_rng(seed)
    jobs = []
    for k in range(n_meshes):
        nv = int(rng.integers(nv_min, nv_max + 1))
        n = int(round(float(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))))
        jobs.append((nv, n, int(rng.integers(0, 2**31 - 1)), int(rng.integers(0, 2**31 - 1)), sdf_n))
    if workers > 1 and n_meshes > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor

        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            meshes = list(ex.map(_star_batch_member, jobs))
    else:
        meshes = [_star_batch_member(j) for j in jobs]
    return BatchWorkload(f"stars{n_meshes}-hybrid-batch", meshes, 2, precision, 100)


def _bilinear_np(g: Grid, x, y):
    """Plain bilinear lookup used only to draw seeds inside a gridded shape."""
    tx = (np.asarray(x) - g.x0) / ((g.x1 - g.x0) / (g.nx - 1))
    ty = (np.asarray(y) - g.y0) / ((g.y1 - g.y0) / (g.ny - 1))
    i = np.clip(np.floor(tx).astype(int), 0, g.nx - 2)
    j = np.clip(np.floor(ty).astype(int), 0, g.ny - 2)
    fx = np.clip(tx - i, 0, 1)
    fy = np.clip(ty - j, 0, 1)
    v = g.values.astype(np.float64)
    a = v[j, i] + fx * (v[j, i + 1] - v[j, i])
    b = v[j + 1, i] + fx * (v[j + 1, i + 1] - v[j + 1, i])
    return a + fy * (b - a)


def lattice_points(kind: str, n_side: int, spacing: float, center=(0.0, 0.0), jitter: float = 0.0, seed: int = 0):
    """Square or hexagonal lattice (exactly representable offsets for the square)."""
    rng = np.random.default_rng(seed)
    pts = []
    for j in range(n_side):
        for i in range(n_side):
            if kind == "square":
                x, y = i * spacing, j * spacing
            else:
                x, y = (i + 0.5 * (j % 2)) * spacing, j * spacing * np.sqrt(3) / 2
            pts.append((x, y))
    p = np.asarray(pts, dtype=np.float64)
    p -= p.mean(0)
    p += np.asarray(center)
    if jitter:
        p += rng.uniform(-jitter, jitter, p.shape)
    return p


def to_fp32_positions(p: np.ndarray) -> np.ndarray:
    """Positions rounded to float32 and widened back (the FP32 mode's inputs)."""
    return p.astype(np.float32).astype(np.float64)
