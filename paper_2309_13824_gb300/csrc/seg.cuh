// seg.cuh -- distance and sign from a closed loop of line segments given
// clockwise (TriMe++ Sec. 3.1), in fixed FP64 formulas (explicit
// round-to-nearest operations) shared by the SDF grid builder and the
// adaptive distance field.
//
// Distance: to the closest segment, the closest point a + t (b - a) with t
// the clamped projection; the smaller segment index wins ties.  Sign:
// negative where (p - p*) . n > 0 with n the segment's inward unit normal
// (right of its direction for a clockwise loop), or, when p* is an end point,
// the sum of the two incident segments' unit normals.
#pragma once
#include "common.cuh"

namespace trime {

__device__ __forceinline__ void seg_dist(const double* xy, int32_t nv, int32_t k, double x, double y, double& d,
                                         double& t) {
    int32_t k1 = k + 1 == nv ? 0 : k + 1;
    double ax = xy[2 * k], ay = xy[2 * k + 1];
    double ex = fsub(xy[2 * k1], ax), ey = fsub(xy[2 * k1 + 1], ay);
    double wx = fsub(x, ax), wy = fsub(y, ay);
    t = fdiv(fadd(fmul(wx, ex), fmul(wy, ey)), fadd(fmul(ex, ex), fmul(ey, ey)));
    if (!(t > 0.0)) t = 0.0;
    if (t > 1.0) t = 1.0;
    double cx = fadd(ax, fmul(t, ex)), cy = fadd(ay, fmul(t, ey));
    double dx = fsub(x, cx), dy = fsub(y, cy);
    d = __dsqrt_rn(fadd(fmul(dx, dx), fmul(dy, dy)));
}

__device__ __forceinline__ void seg_normal(const double* xy, int32_t nv, int32_t k, double& nx, double& ny) {
    int32_t k1 = k + 1 == nv ? 0 : k + 1;
    double dx = fsub(xy[2 * k1], xy[2 * k]), dy = fsub(xy[2 * k1 + 1], xy[2 * k + 1]);
    double L = __dsqrt_rn(fadd(fmul(dx, dx), fmul(dy, dy)));
    nx = fdiv(dy, L);
    ny = fdiv(-dx, L);
}

// cell grid of about the mean segment length over a box (Sec. 3.1)
struct SegGrid {
    double x0, y0, cw, ch;  // cell grid origin and cell size
    int32_t gx, gy;
    double diag;
};

__device__ __forceinline__ int cell_x(const SegGrid& G, double x) {
    double f = floor((x - G.x0) / G.cw);
    return f < 0.0 ? 0 : (f > (double)(G.gx - 1) ? G.gx - 1 : (int)f);
}
__device__ __forceinline__ int cell_y(const SegGrid& G, double y) {
    double f = floor((y - G.y0) / G.ch);
    return f < 0.0 ? 0 : (f > (double)(G.gy - 1) ? G.gy - 1 : (int)f);
}

// signed distance at (x, y) given its closest segment k, the projection
// parameter t and the distance d
__device__ __forceinline__ double seg_signed(const double* xy, int32_t nv, int32_t k, double t, double d, double x,
                                             double y) {
    int32_t k1 = k + 1 == nv ? 0 : k + 1;
    double ax = xy[2 * k], ay = xy[2 * k + 1];
    double ex = fsub(xy[2 * k1], ax), ey = fsub(xy[2 * k1 + 1], ay);
    double cx = fadd(ax, fmul(t, ex)), cy = fadd(ay, fmul(t, ey));
    double nxv, nyv;
    seg_normal(xy, nv, k, nxv, nyv);
    if (t == 0.0 || t == 1.0) {
        int other = t == 0.0 ? (k == 0 ? nv - 1 : k - 1) : k1;
        double mx, my;
        seg_normal(xy, nv, other, mx, my);
        nxv = fadd(nxv, mx);
        nyv = fadd(nyv, my);
    }
    double s = fadd(fmul(fsub(x, cx), nxv), fmul(fsub(y, cy), nyv));
    return s > 0.0 ? -d : d;
}

// the signed distance at (x, y) by a search over every segment
__device__ __forceinline__ double seg_sdf_point(const double* xy, int32_t nv, double x, double y) {
    double best = INFINITY, bt = 0.0;
    int32_t bk = 0;
    for (int32_t k = 0; k < nv; k++) {
        double d, t;
        seg_dist(xy, nv, k, x, y, d, t);
        if (d < best) {
            best = d;
            bk = k;
            bt = t;
        }
    }
    return seg_signed(xy, nv, bk, bt, best, x, y);
}

// the signed distance at (x, y) from the candidate list of its cell (each
// cell's list holds the closest segment of every point of the cell); ties
// go to the smaller index, so the value equals the search over every segment
__device__ __forceinline__ double seg_sdf_cand(const double* xy, int32_t nv, const SegGrid& G, const int32_t* cstart,
                                               const int32_t* cand, double x, double y) {
    int c = cell_y(G, y) * G.gx + cell_x(G, x);
    double best = INFINITY, bt = 0.0;
    int bk = 0x7fffffff;
    for (int u = cstart[c]; u < cstart[c + 1]; u++) {
        int k = cand[u];
        double d, t;
        seg_dist(xy, nv, k, x, y, d, t);
        if (d < best || (d == best && k < bk)) {
            best = d;
            bk = k;
            bt = t;
        }
    }
    if (bk >= nv) return __longlong_as_double(0x7ff8000000000000ll);  // no candidate: cannot happen
    return seg_signed(xy, nv, bk, bt, best, x, y);
}

// Device candidate lists of a segment loop over a box, built by
// seg_index_build (sdf.cu) and released by seg_index_free.
struct SegIndex {
    SegGrid G{};
    int32_t *cnt = nullptr, *start = nullptr, *cur = nullptr, *list = nullptr, *tmp = nullptr;
    int32_t *ncand = nullptr, *cstart = nullptr, *cand = nullptr;
    double* rad = nullptr;
};
// hxy: the loop on the host (validated: finite, no zero-length segment);
// dxy: the same on the device.  Returns a TRIME_ status.
int seg_index_build(const double* hxy, const double* dxy, int64_t nv, double x0, double y0, double x1, double y1,
                    SegIndex* out, cudaStream_t st);
void seg_index_free(SegIndex* s);

}  // namespace trime
