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


_SEG_TREES = {}


def _segment_samples(verts_cw, h):
    """kd-tree of points spaced h/4 along every segment, and their segment."""
    from scipy.spatial import cKDTree

    key = (verts_cw.tobytes(), float(h))
    if key not in _SEG_TREES:
        a = verts_cw
        b = np.roll(verts_cw, -1, axis=0)
        seg_len = np.hypot(*(b - a).T)
        k_per = np.maximum(2, np.ceil(seg_len / (h / 4)).astype(int))
        samples, owner = [], []
        for s in range(len(a)):
            t = np.linspace(0, 1, k_per[s], endpoint=False)
            samples.append(a[s] + t[:, None] * (b[s] - a[s]))
            owner.append(np.full(k_per[s], s))
        samples = np.concatenate(samples)
        _SEG_TREES.clear()
        _SEG_TREES[key] = (cKDTree(samples), np.concatenate(owner))
    return _SEG_TREES[key]


def _polygon_sdf_rows(args):
    verts_cw, n, box, j0, j1 = args
    x0, y0, x1, y1 = box
    xs = x0 + np.arange(n) * ((x1 - x0) / (n - 1))
    ys = y0 + np.arange(j0, j1) * ((y1 - y0) / (n - 1))
    X, Y = np.meshgrid(xs, ys)
    P = np.stack([X.ravel(), Y.ravel()], 1)
    a = verts_cw
    b = np.roll(verts_cw, -1, axis=0)
    h = (x1 - x0) / (n - 1)
    tree, owner = _segment_samples(verts_cw, h)
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
    return np.where(inside, -best, best).reshape(X.shape).astype(np.float32)


def polygon_sdf_grid(verts_cw, n: int, box=BOX, workers: int = 0) -> Grid:
    """Signed distance to a star polygon: nearest-segment distance, sign from
    the radial inside test (the polygon is star-shaped around the origin).
    Rows are computed in blocks, in `workers` spawned processes if > 1."""
    step = max(1, (1 << 18) // n)
    jobs = [(verts_cw, n, box, j, min(n, j + step)) for j in range(0, n, step)]
    if workers > 1 and len(jobs) > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor

        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            rows = list(ex.map(_polygon_sdf_rows, jobs))
    else:
        rows = [_polygon_sdf_rows(j) for j in jobs]
    return Grid(np.ascontiguousarray(np.concatenate(rows, 0), dtype=np.float32), *box)


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


def _seg_dist(P, A, B):
    """Distance from points P (m, 2) to segments A-B (broadcast)."""
    e = B - A
    t = np.clip(((P - A) * e).sum(-1) / (e * e).sum(-1), 0.0, 1.0)
    return np.hypot(*np.moveaxis(P - (A + t[..., None] * e), -1, 0))


def star_lfs(verts_cw):
    """Local thickness at each vertex: distance to the nearest segment not
    incident to it."""
    nv = len(verts_cw)
    a = verts_cw
    b = np.roll(verts_cw, -1, axis=0)
    d = _seg_dist(verts_cw[:, None, :], a[None, :, :], b[None, :, :])  # (vertex, segment)
    idx = np.arange(nv)
    d[idx, idx] = np.inf            # segment (v, v+1)
    d[idx, (idx - 1) % nv] = np.inf  # segment (v-1, v)
    return d.min(1)


def star_sizing_grid(verts_cw, n: int, lo: float = 2e-4, hi: float = 1e-2, grad: float = 0.1,
                     box=BOX) -> Grid:
    """Curvature-adaptive sizing h(x) = clamp(min_s grad |x - v_s| + t(v_s), lo, hi)
    over the polygon's vertices v_s, sampled on n^2 nodes, where the vertex
    size t(v) is proportional to the local thickness lfs(v) and scaled so that
    the narrowest vertex gets lo: the sizes span [lo, hi]."""
    from scipy.spatial import cKDTree

    t = star_lfs(verts_cw)
    t = t * (lo / t.min())
    X, Y = _node_grid(n, box)
    P = np.stack([X.ravel(), Y.ravel()], 1)
    # min_s grad |x - v_s| + t_s over the k nearest vertices, exact wherever the
    # k-th nearest cannot win (grad d_k + min t >= the minimum found); the
    # remaining nodes are evaluated against every vertex
    k = min(16, len(verts_cw))
    d, idx = cKDTree(verts_cw).query(P, k=k)
    d = d.reshape(len(P), k)
    idx = idx.reshape(len(P), k)
    h = (grad * d + t[idx]).min(1)
    open_ = np.nonzero(grad * d[:, -1] + t.min() < h)[0]
    for c in range(0, len(open_), 1 << 14):
        q = P[open_[c:c + (1 << 14)]]
        dd = np.hypot(q[:, None, 0] - verts_cw[None, :, 0], q[:, None, 1] - verts_cw[None, :, 1])
        h[open_[c:c + (1 << 14)]] = (grad * dd + t[None, :]).min(1)
    h = np.clip(h, lo, hi).reshape(X.shape)
    return Grid(np.ascontiguousarray(h, dtype=np.float32), *box)


def _density_grid_chunk(args):
    sdf, siz, n, seed_seq = args
    rng = np.random.default_rng(seed_seq)
    v = siz.values.astype(np.float64)
    hmin = np.minimum(np.minimum(v[:-1, :-1], v[:-1, 1:]), np.minimum(v[1:, :-1], v[1:, 1:])).ravel()
    cdf = np.cumsum(1.0 / hmin**2)
    cdf /= cdf[-1]
    dx = (siz.x1 - siz.x0) / (siz.nx - 1)
    dy = (siz.y1 - siz.y0) / (siz.ny - 1)
    ncx = siz.nx - 1
    out = []
    got = 0
    while got < n:
        m = max(1 << 16, 3 * (n - got))
        c = np.minimum(np.searchsorted(cdf, rng.uniform(0, 1, m), side="right"), len(cdf) - 1)
        ci, cj = c % ncx, c // ncx
        x = siz.x0 + (ci + rng.uniform(0, 1, m)) * dx
        y = siz.y0 + (cj + rng.uniform(0, 1, m)) * dy
        keep = rng.uniform(0, 1, m) < (hmin[c] / _bilinear_np(siz, x, y)) ** 2
        x, y = x[keep], y[keep]
        inside = _bilinear_np(sdf, x, y) < 0
        p = np.stack([x[inside], y[inside]], 1)
        out.append(p)
        got += len(p)
    return np.concatenate(out)[:n]


def density_in_grid(sdf: Grid, siz: Grid, n: int, seed: int, workers: int = 0):
    """n points inside {sdf < 0} with density proportional to 1/h^2 for the
    bilinear sizing grid h: cells of the sizing grid are drawn with weight
    area / hmin_cell^2 (hmin_cell = smallest corner value, a lower bound of h
    in the cell), a point uniform in the cell is kept with probability
    (hmin_cell / h(p))^2 and if sdf(p) < 0 (exact rejection sampling).  Points
    come in blocks of 2^20 with their own seeds (numpy SeedSequence), so the
    result does not depend on `workers`."""
    block = 1 << 20
    counts = [min(block, n - k) for k in range(0, n, block)]
    seqs = np.random.SeedSequence(seed).spawn(len(counts))
    jobs = [(sdf, siz, c, q) for c, q in zip(counts, seqs)]
    if workers > 1 and len(jobs) > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor

        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_density_grid_chunk, jobs))
    else:
        parts = [_density_grid_chunk(j) for j in jobs]
    if not parts:
        return np.zeros((0, 2))
    return np.ascontiguousarray(np.concatenate(parts), dtype=np.float64)


def star_workload(n: int, nv: int = 500, seed: int = 2, sdf_n: int = 4096, siz_n: int = 1024,
                  precision: int = 1, workers: int = 0) -> Workload:
    """Random star polygon (nv vertices at angles 2 pi k / nv, radii
    U[0.4, 1]), exact segment SDF on sdf_n^2, curvature-adaptive sizing in
    [2e-4, 1e-2] on siz_n^2 (star_sizing_grid), n points ~ 1/h^2 (seed + 1)."""
    verts = star_polygon(nv, 0.4, 1.0, seed)
    sdf = polygon_sdf_grid(verts, sdf_n, workers=workers)
    siz = star_sizing_grid(verts, siz_n)
    pts = density_in_grid(sdf, siz, n, seed + 1, workers=workers)
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
