// adf.cu -- the adaptive distance field of TriMe++ Sec. 3.7 (Fig. 17; App. B
// T_depth, fac_Etol): one quadtree per listed grid cell, built top-down.  A
// node's four corners hold the exact signed distance to the segment loop;
// the node splits into four children when the bilinear values at its four
// edge midpoints and its centre differ from the exact distances there by
// more than the cell's tolerance, up to a maximum depth.  Evaluation descends
// to the leaf holding the point and interpolates bilinearly.
//
// GB300 layout: the trees are built level by level over all cells at once
// (one thread per node tests it; a scan numbers the children; one thread per
// split node writes its four children), so nodes come out in level order,
// each parent's children consecutive and in their parents' order.  Node
// arrays: v[4n] corners (v00, v10, v01, v11) FP64, child[n] (first child or
// -1), root[n] (index into the cell list), lev[3n] (level, ix, iy).  Every
// coordinate and comparison uses fixed FP64 formulas (explicit
// round-to-nearest operations), so the trees do not depend on the schedule.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "seg.cuh"
#include "trime.h"

namespace trime {

struct AdfGrid {
    double x0, y0, dx, dy;
    int32_t ncx, ncy;
};

// coordinate of corner index i at level L of a cell starting at c0: c0 + i (w 2^-L)
__device__ __forceinline__ double adf_coord(double c0, double w, int32_t i, int32_t L) {
    return fadd(c0, fmul((double)i, fmul(w, fdiv(1.0, (double)(1 << L)))));
}

__device__ __forceinline__ void cell_origin(const AdfGrid& G, int32_t c, double& cx0, double& cy0) {
    cx0 = fadd(G.x0, fmul((double)(c % G.ncx), G.dx));
    cy0 = fadd(G.y0, fmul((double)(c / G.ncx), G.dy));
}

__global__ void k_adf_cellroot(const int32_t* cells, int32_t ncells, int32_t* cellroot) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < ncells) cellroot[cells[r]] = r;
}

__global__ void k_adf_roots(const double* xy, int32_t nv, SegGrid S, const int32_t* cstart, const int32_t* cand,
                            AdfGrid G, const int32_t* cells, int32_t ncells, double* v, int32_t* child, int32_t* root,
                            int32_t* lev) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ncells) return;
    double cx0, cy0;
    cell_origin(G, cells[r], cx0, cy0);
    double xa = adf_coord(cx0, G.dx, 0, 0), xb = adf_coord(cx0, G.dx, 1, 0);
    double ya = adf_coord(cy0, G.dy, 0, 0), yb = adf_coord(cy0, G.dy, 1, 0);
    v[4 * r] = seg_sdf_cand(xy, nv, S, cstart, cand, xa, ya);
    v[4 * r + 1] = seg_sdf_cand(xy, nv, S, cstart, cand, xb, ya);
    v[4 * r + 2] = seg_sdf_cand(xy, nv, S, cstart, cand, xa, yb);
    v[4 * r + 3] = seg_sdf_cand(xy, nv, S, cstart, cand, xb, yb);
    child[r] = -1;
    root[r] = r;
    lev[3 * r] = lev[3 * r + 1] = lev[3 * r + 2] = 0;
}

// nodes [lo, lo + count) of level L: exact distances at the bottom, top,
// left, right midpoints and the centre; split flag
__global__ void k_adf_test(const double* xy, int32_t nv, SegGrid S, const int32_t* cstart, const int32_t* cand,
                           AdfGrid G, const int32_t* cells, const double* tol, const double* v, const int32_t* root,
                           const int32_t* lev, int64_t lo, int32_t count, int32_t* flag, double* s5) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    int64_t n = lo + k;
    int32_t r = root[n], L = lev[3 * n], ix = lev[3 * n + 1], iy = lev[3 * n + 2];
    double cx0, cy0;
    cell_origin(G, cells[r], cx0, cy0);
    double xa = adf_coord(cx0, G.dx, 2 * ix, L + 1), xm = adf_coord(cx0, G.dx, 2 * ix + 1, L + 1);
    double xb = adf_coord(cx0, G.dx, 2 * ix + 2, L + 1);
    double ya = adf_coord(cy0, G.dy, 2 * iy, L + 1), ym = adf_coord(cy0, G.dy, 2 * iy + 1, L + 1);
    double yb = adf_coord(cy0, G.dy, 2 * iy + 2, L + 1);
    double s[5];
    s[0] = seg_sdf_cand(xy, nv, S, cstart, cand, xm, ya);
    s[1] = seg_sdf_cand(xy, nv, S, cstart, cand, xm, yb);
    s[2] = seg_sdf_cand(xy, nv, S, cstart, cand, xa, ym);
    s[3] = seg_sdf_cand(xy, nv, S, cstart, cand, xb, ym);
    s[4] = seg_sdf_cand(xy, nv, S, cstart, cand, xm, ym);
    double v00 = v[4 * n], v10 = v[4 * n + 1], v01 = v[4 * n + 2], v11 = v[4 * n + 3];
    double p[5] = {fmul(fadd(v00, v10), 0.5), fmul(fadd(v01, v11), 0.5), fmul(fadd(v00, v01), 0.5),
                   fmul(fadd(v10, v11), 0.5), fmul(fadd(fadd(v00, v10), fadd(v01, v11)), 0.25)};
    double err = 0.0;
    for (int q = 0; q < 5; q++) err = fmax(err, fabs(fsub(p[q], s[q])));
    flag[k] = err > tol[r] ? 1 : 0;
    for (int q = 0; q < 5; q++) s5[5 * (int64_t)k + q] = s[q];
}

// the four children of every split node of [lo, lo + count), numbered from base
__global__ void k_adf_split(double* v, int32_t* child, int32_t* root, int32_t* lev, int64_t lo, int32_t count,
                            const int32_t* flag, const int32_t* off, const double* s5, int64_t base) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count || !flag[k]) return;
    int64_t n = lo + k, c = base + 4 * (int64_t)off[k];
    child[n] = (int32_t)c;
    const double* s = s5 + 5 * (int64_t)k;
    double v00 = v[4 * n], v10 = v[4 * n + 1], v01 = v[4 * n + 2], v11 = v[4 * n + 3];
    // quadrants (0,0), (1,0), (0,1), (1,1): corners from the parent's corners,
    // the midpoints (bottom s0, top s1, left s2, right s3) and the centre s4
    const double cv[4][4] = {{v00, s[0], s[2], s[4]}, {s[0], v10, s[4], s[3]}, {s[2], s[4], v01, s[1]},
                             {s[4], s[3], s[1], v11}};
    int32_t L = lev[3 * n], ix = lev[3 * n + 1], iy = lev[3 * n + 2];
    for (int q = 0; q < 4; q++) {
        int64_t m = c + q;
        for (int t = 0; t < 4; t++) v[4 * m + t] = cv[q][t];
        child[m] = -1;
        root[m] = root[n];
        lev[3 * m] = L + 1;
        lev[3 * m + 1] = 2 * ix + (q & 1);
        lev[3 * m + 2] = 2 * iy + (q >> 1);
    }
}

__global__ void k_adf_eval(AdfGrid G, const int32_t* cellroot, const int32_t* cells, const double* v,
                           const int32_t* child, const int32_t* lev, const double* pts, int64_t np, double* out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= np) return;
    double x = pts[2 * q], y = pts[2 * q + 1];
    double fi = floor(fdiv(fsub(x, G.x0), G.dx)), fj = floor(fdiv(fsub(y, G.y0), G.dy));
    int32_t i = !(fi >= 0.0) ? 0 : (fi > (double)(G.ncx - 1) ? G.ncx - 1 : (int32_t)fi);
    int32_t j = !(fj >= 0.0) ? 0 : (fj > (double)(G.ncy - 1) ? G.ncy - 1 : (int32_t)fj);
    int32_t r = cellroot[(int64_t)j * G.ncx + i];
    if (r < 0) {
        out[q] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    double cx0, cy0;
    cell_origin(G, cells[r], cx0, cy0);
    int64_t k = r;
    for (int guard = 0; child[k] >= 0 && guard < 16; guard++) {
        int32_t L = lev[3 * k], ix = lev[3 * k + 1], iy = lev[3 * k + 2];
        double xm = adf_coord(cx0, G.dx, 2 * ix + 1, L + 1), ym = adf_coord(cy0, G.dy, 2 * iy + 1, L + 1);
        k = child[k] + (y >= ym ? 2 : 0) + (x >= xm ? 1 : 0);
    }
    int32_t L = lev[3 * k], ix = lev[3 * k + 1], iy = lev[3 * k + 2];
    double sc = fdiv(1.0, (double)(1 << L));
    double wx = fmul(G.dx, sc), wy = fmul(G.dy, sc);
    double fx = fdiv(fsub(x, adf_coord(cx0, G.dx, ix, L)), wx), fy = fdiv(fsub(y, adf_coord(cy0, G.dy, iy, L)), wy);
    fx = fx < 0.0 ? 0.0 : (fx > 1.0 ? 1.0 : fx);
    fy = fy < 0.0 ? 0.0 : (fy > 1.0 ? 1.0 : fy);
    const double* c = v + 4 * k;
    double va = fadd(c[0], fmul(fx, fsub(c[1], c[0]))), vb = fadd(c[2], fmul(fx, fsub(c[3], c[2])));
    out[q] = fadd(va, fmul(fy, fsub(vb, va)));
}

__global__ void k_sdf_points(const double* xy, int32_t nv, const double* pts, int64_t np, double* out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < np) out[q] = seg_sdf_point(xy, nv, pts[2 * q], pts[2 * q + 1]);
}

}  // namespace trime

using namespace trime;

struct adf_s {
    AdfGrid G{};
    int32_t nv = 0, ncells = 0, levels = 0;
    double* xy = nullptr;
    int32_t* cells = nullptr;
    double* tol = nullptr;
    int32_t* cellroot = nullptr;
    int64_t n = 0, cap = 0;
    double* v = nullptr;
    int32_t *child = nullptr, *root = nullptr, *lev = nullptr;
};

// the loop's vertices finite and its segments of positive length
static int check_loop(const double* xy, int64_t nv) {
    for (int64_t k = 0; k < nv; k++) {
        int64_t k1 = k + 1 == nv ? 0 : k + 1;
        if (!std::isfinite(xy[2 * k]) || !std::isfinite(xy[2 * k + 1]))
            return set_error(TRIME_EINVAL, "polygon coordinates must be finite");
        if (!(std::hypot(xy[2 * k1] - xy[2 * k], xy[2 * k1 + 1] - xy[2 * k + 1]) > 0.0))
            return set_error(TRIME_EINVAL, "zero-length segment");
    }
    return TRIME_OK;
}

static void adf_release(adf_s* a) {
    if (!a) return;
    for (void* p : {(void*)a->xy, (void*)a->cells, (void*)a->tol, (void*)a->cellroot, (void*)a->v, (void*)a->child,
                    (void*)a->root, (void*)a->lev})
        if (p) cudaFree(p);
    delete a;
}

#define ADF_TRY(x)                                                                                  \
    do {                                                                                            \
        cudaError_t e_ = (x);                                                                       \
        if (e_ != cudaSuccess) {                                                                    \
            rc = set_error(TRIME_ECUDA, (std::string(#x) + ": " + cudaGetErrorString(e_)).c_str()); \
            goto done;                                                                              \
        }                                                                                           \
    } while (0)

// grow the node arrays to hold need nodes, keeping the first a->n
static int adf_grow(adf_s* a, int64_t need, cudaStream_t st) {
    if (need <= a->cap) return TRIME_OK;
    int64_t cap = std::max<int64_t>(a->cap, 1024);
    while (cap < need) cap *= 2;
    if (cap > ((int64_t)1 << 30)) return set_error(TRIME_ECAPACITY, "ADF: more than 2^30 nodes");
    int rc = TRIME_OK;
    double* v = nullptr;
    int32_t *child = nullptr, *root = nullptr, *lev = nullptr;
    ADF_TRY(cudaMalloc(&v, sizeof(double) * 4 * (size_t)cap));
    ADF_TRY(cudaMalloc(&child, sizeof(int32_t) * (size_t)cap));
    ADF_TRY(cudaMalloc(&root, sizeof(int32_t) * (size_t)cap));
    ADF_TRY(cudaMalloc(&lev, sizeof(int32_t) * 3 * (size_t)cap));
    if (a->n > 0) {
        ADF_TRY(cudaMemcpyAsync(v, a->v, sizeof(double) * 4 * (size_t)a->n, cudaMemcpyDeviceToDevice, st));
        ADF_TRY(cudaMemcpyAsync(child, a->child, sizeof(int32_t) * (size_t)a->n, cudaMemcpyDeviceToDevice, st));
        ADF_TRY(cudaMemcpyAsync(root, a->root, sizeof(int32_t) * (size_t)a->n, cudaMemcpyDeviceToDevice, st));
        ADF_TRY(cudaMemcpyAsync(lev, a->lev, sizeof(int32_t) * 3 * (size_t)a->n, cudaMemcpyDeviceToDevice, st));
        ADF_TRY(cudaStreamSynchronize(st));
    }
    for (void* p : {(void*)a->v, (void*)a->child, (void*)a->root, (void*)a->lev})
        if (p) cudaFree(p);
    a->v = v;
    a->child = child;
    a->root = root;
    a->lev = lev;
    a->cap = cap;
    return TRIME_OK;
done:
    for (void* p : {(void*)v, (void*)child, (void*)root, (void*)lev})
        if (p) cudaFree(p);
    return rc;
}

extern "C" int mesh_adf_build(const double* xy, int64_t nv, double x0, double y0, double x1, double y1, int32_t nx,
                              int32_t ny, const int32_t* cells, const double* tol, int32_t ncells, int32_t max_depth,
                              adf_t** out, void* cuda_stream) {
    if (!out) return set_error(TRIME_EINVAL, "NULL output handle");
    *out = nullptr;
    if (!xy || (ncells > 0 && (!cells || !tol))) return set_error(TRIME_EINVAL, "NULL pointer");
    if (nv < 3 || nv > (int64_t)1 << 26) return set_error(TRIME_EINVAL, "need 3 .. 2^26 vertices");
    if (nx < 2 || ny < 2 || (int64_t)(nx - 1) * (ny - 1) > ((int64_t)1 << 31) - 1)
        return set_error(TRIME_EINVAL, "grid must have at least 2 nodes per side and < 2^31 cells");
    if (!(x1 > x0) || !(y1 > y0) || !std::isfinite(x0) || !std::isfinite(x1) || !std::isfinite(y0) ||
        !std::isfinite(y1))
        return set_error(TRIME_EINVAL, "bad grid box");
    if (ncells < 0 || max_depth < 0 || max_depth > 14) return set_error(TRIME_EINVAL, "need ncells >= 0, 0 <= max_depth <= 14");
    if (int rc0 = check_loop(xy, nv)) return rc0;
    int64_t ncell_all = (int64_t)(nx - 1) * (ny - 1);
    {
        std::vector<uint8_t> seen((size_t)ncell_all, 0);
        for (int32_t r = 0; r < ncells; r++) {
            if (cells[r] < 0 || cells[r] >= ncell_all || seen[(size_t)cells[r]])
                return set_error(TRIME_EINVAL, "cells must be distinct grid cells");
            seen[(size_t)cells[r]] = 1;
            if (!(tol[r] >= 0.0) || !std::isfinite(tol[r])) return set_error(TRIME_EINVAL, "tolerances must be finite, >= 0");
        }
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    adf_s* a = new adf_s;
    a->G.x0 = x0;
    a->G.y0 = y0;
    a->G.dx = (x1 - x0) / (double)(nx - 1);
    a->G.dy = (y1 - y0) / (double)(ny - 1);
    a->G.ncx = nx - 1;
    a->G.ncy = ny - 1;
    a->nv = (int32_t)nv;
    a->ncells = ncells;
    int rc = TRIME_OK;
    int32_t *flag = nullptr, *off = nullptr, *tmp = nullptr;
    double* s5 = nullptr;
    SegIndex SI;
    int32_t fcap = 0;
    int64_t lo = 0, hi = ncells;
    ADF_TRY(cudaMalloc(&a->xy, sizeof(double) * 2 * (size_t)nv));
    ADF_TRY(cudaMalloc(&a->cells, sizeof(int32_t) * (size_t)std::max(ncells, 1)));
    ADF_TRY(cudaMalloc(&a->tol, sizeof(double) * (size_t)std::max(ncells, 1)));
    ADF_TRY(cudaMalloc(&a->cellroot, sizeof(int32_t) * (size_t)ncell_all));
    ADF_TRY(cudaMemcpyAsync(a->xy, xy, sizeof(double) * 2 * (size_t)nv, cudaMemcpyHostToDevice, st));
    if (ncells > 0) {
        ADF_TRY(cudaMemcpyAsync(a->cells, cells, sizeof(int32_t) * (size_t)ncells, cudaMemcpyHostToDevice, st));
        ADF_TRY(cudaMemcpyAsync(a->tol, tol, sizeof(double) * (size_t)ncells, cudaMemcpyHostToDevice, st));
    }
    ADF_TRY(cudaMemsetAsync(a->cellroot, 0xff, sizeof(int32_t) * (size_t)ncell_all, st));
    // exact distances from the candidate lists of a segment cell grid over the box
    if ((rc = seg_index_build(xy, a->xy, nv, x0, y0, x1, y1, &SI, st))) goto done;
    if ((rc = adf_grow(a, std::max<int64_t>(4 * (int64_t)ncells, 1024), st))) goto done;
    if (ncells > 0) {
        k_adf_cellroot<<<(ncells + 255) / 256, 256, 0, st>>>(a->cells, ncells, a->cellroot);
        k_adf_roots<<<(ncells + 127) / 128, 128, 0, st>>>(a->xy, a->nv, SI.G, SI.cstart, SI.cand, a->G, a->cells,
                                                         ncells, a->v, a->child, a->root, a->lev);
        ADF_TRY(cudaGetLastError());
    }
    a->n = ncells;
    a->levels = ncells > 0 ? 1 : 0;
    for (int32_t L = 0; L < max_depth && hi > lo; L++) {
        int32_t count = (int32_t)(hi - lo);
        if (count > fcap) {
            for (void* p : {(void*)flag, (void*)off, (void*)tmp, (void*)s5})
                if (p) cudaFree(p);
            flag = off = tmp = nullptr;
            s5 = nullptr;
            fcap = std::max(count, 1024);
            ADF_TRY(cudaMalloc(&flag, sizeof(int32_t) * (size_t)fcap));
            ADF_TRY(cudaMalloc(&off, sizeof(int32_t) * ((size_t)fcap + 1)));
            ADF_TRY(cudaMalloc(&tmp, sizeof(int32_t) * ((size_t)fcap / 4096 + 2)));
            ADF_TRY(cudaMalloc(&s5, sizeof(double) * 5 * (size_t)fcap));
        }
        k_adf_test<<<(count + 127) / 128, 128, 0, st>>>(a->xy, a->nv, SI.G, SI.cstart, SI.cand, a->G, a->cells,
                                                        a->tol, a->v, a->root, a->lev, lo, count, flag, s5);
        launch_scan(flag, off, count, tmp, st);
        ADF_TRY(cudaGetLastError());
        int32_t nsplit = 0;
        ADF_TRY(cudaMemcpyAsync(&nsplit, off + count, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        ADF_TRY(cudaStreamSynchronize(st));
        if (nsplit == 0) break;
        if ((rc = adf_grow(a, hi + 4 * (int64_t)nsplit, st))) goto done;
        k_adf_split<<<(count + 127) / 128, 128, 0, st>>>(a->v, a->child, a->root, a->lev, lo, count, flag, off, s5,
                                                         hi);
        ADF_TRY(cudaGetLastError());
        lo = hi;
        hi += 4 * (int64_t)nsplit;
        a->n = hi;
        a->levels = L + 2;
    }
    ADF_TRY(cudaStreamSynchronize(st));
done:
    cudaStreamSynchronize(st);
    seg_index_free(&SI);
    for (void* p : {(void*)flag, (void*)off, (void*)tmp, (void*)s5})
        if (p) cudaFree(p);
    if (rc) {
        adf_release(a);
        return rc;
    }
    *out = a;
    return TRIME_OK;
}

extern "C" int mesh_adf_size(const adf_t* a, int64_t* n_nodes, int32_t* n_levels) {
    if (!a || !n_nodes || !n_levels) return set_error(TRIME_EINVAL, "NULL argument");
    *n_nodes = a->n;
    *n_levels = a->levels;
    return TRIME_OK;
}

extern "C" int mesh_adf_export(const adf_t* a, double* v, int32_t* child, int32_t* root, int32_t* lev, int64_t cap,
                               int64_t* n_out) {
    if (!a || !v || !child || !root || !lev || !n_out) return set_error(TRIME_EINVAL, "NULL argument");
    *n_out = a->n;
    if (cap < a->n) return set_error(TRIME_ECAPACITY, "ADF export buffers too small");
    if (a->n == 0) return TRIME_OK;
    int rc = TRIME_OK;
    ADF_TRY(cudaMemcpy(v, a->v, sizeof(double) * 4 * (size_t)a->n, cudaMemcpyDeviceToHost));
    ADF_TRY(cudaMemcpy(child, a->child, sizeof(int32_t) * (size_t)a->n, cudaMemcpyDeviceToHost));
    ADF_TRY(cudaMemcpy(root, a->root, sizeof(int32_t) * (size_t)a->n, cudaMemcpyDeviceToHost));
    ADF_TRY(cudaMemcpy(lev, a->lev, sizeof(int32_t) * 3 * (size_t)a->n, cudaMemcpyDeviceToHost));
done:
    return rc;
}

static bool on_device(const void* p) {
    cudaPointerAttributes at;
    bool dev = cudaPointerGetAttributes(&at, p) == cudaSuccess &&
               (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    return dev;
}

// run a per-point kernel on host or device buffers of n (x, y) pairs
template <typename F>
static int points_call(const double* pts, int64_t np, double* out, cudaStream_t st, F launch) {
    int rc = TRIME_OK;
    bool din = on_device(pts), dout = on_device(out);
    double *dp = nullptr, *dv = nullptr;
    if (din) dp = const_cast<double*>(pts);
    else {
        ADF_TRY(cudaMalloc(&dp, sizeof(double) * 2 * (size_t)np));
        ADF_TRY(cudaMemcpyAsync(dp, pts, sizeof(double) * 2 * (size_t)np, cudaMemcpyHostToDevice, st));
    }
    if (dout) dv = out;
    else ADF_TRY(cudaMalloc(&dv, sizeof(double) * (size_t)np));
    launch(dp, dv);
    ADF_TRY(cudaGetLastError());
    if (!dout) ADF_TRY(cudaMemcpyAsync(out, dv, sizeof(double) * (size_t)np, cudaMemcpyDeviceToHost, st));
    ADF_TRY(cudaStreamSynchronize(st));
done:
    if (dp && !din) cudaFree(dp);
    if (dv && !dout) cudaFree(dv);
    return rc;
}

extern "C" int mesh_adf_eval(const adf_t* a, const double* pts, int64_t np, double* out, void* cuda_stream) {
    if (!a || (np > 0 && (!pts || !out))) return set_error(TRIME_EINVAL, "NULL argument");
    if (np < 0 || np > ((int64_t)1 << 34)) return set_error(TRIME_EINVAL, "bad point count");
    if (np == 0) return TRIME_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    return points_call(pts, np, out, st, [&](const double* dp, double* dv) {
        k_adf_eval<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(a->G, a->cellroot, a->cells, a->v, a->child, a->lev,
                                                                 dp, np, dv);
    });
}

extern "C" void mesh_adf_destroy(adf_t* a) { adf_release(a); }

extern "C" int mesh_segment_sdf_points(const double* xy, int64_t nv, const double* pts, int64_t np, double* out,
                                       void* cuda_stream) {
    if (!xy || (np > 0 && (!pts || !out))) return set_error(TRIME_EINVAL, "NULL pointer");
    if (nv < 3 || nv > (int64_t)1 << 26) return set_error(TRIME_EINVAL, "need 3 .. 2^26 vertices");
    if (np < 0 || np > ((int64_t)1 << 34)) return set_error(TRIME_EINVAL, "bad point count");
    if (int rc0 = check_loop(xy, nv)) return rc0;
    if (np == 0) return TRIME_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc = TRIME_OK;
    double* dxy = nullptr;
    ADF_TRY(cudaMalloc(&dxy, sizeof(double) * 2 * (size_t)nv));
    ADF_TRY(cudaMemcpyAsync(dxy, xy, sizeof(double) * 2 * (size_t)nv, cudaMemcpyHostToDevice, st));
    rc = points_call(pts, np, out, st, [&](const double* dp, double* dv) {
        k_sdf_points<<<(unsigned)((np + 127) / 128), 128, 0, st>>>(dxy, (int32_t)nv, dp, np, dv);
    });
done:
    if (dxy) {
        cudaStreamSynchronize(st);
        cudaFree(dxy);
    }
    return rc;
}
