// common.cuh -- shared device types and the fixed floating-point formulas of
// the meshing iteration (TriMe++, arXiv 2309.13824).
//
// Decisions that select triangles (bounded-region membership, Tests 1-3 of
// Sec. 4.1, geometry-cell lookup) are evaluated by fixed FP64 formulas written
// with explicit round-to-nearest intrinsics, so the compiler never contracts
// them into fused multiply-adds; every other quantity may use FMAs freely.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace trime {

constexpr int kWarp = 32;
constexpr int kRingCap = 64;  // edges per cell: 16 or 32 in a warp's lanes, up to 64 in the serial pass
constexpr int kWarm = 8;      // neighbours of the previous triangulation a cell starts from
constexpr double kRT = 0.70710678118654752440;  // double nearest sqrt(2)/2

enum : uint8_t { CELL_INNER = 0, CELL_BOUNDARY = 1, CELL_OUTER = 2 };
enum : uint8_t { PT_INNER = 0, PT_BOUNDARY = 1, PT_OUTSIDE = 2 };

// bounding-edge labels in a ring: bisectors carry the neighbour's sorted slot (>= 0)
__host__ __device__ constexpr int32_t oct_label(int k) { return -1 - k; }   // -1..-8
__host__ __device__ constexpr int32_t box_label(int b) { return -9 - b; }   // -9..-12 (L,R,B,T)
constexpr int32_t kNoLabel = -1000;  // an empty entry of a previous-neighbour row

struct DevGrid {
    int32_t nx, ny;
    double x0, y0, x1, y1, dx, dy;
    const float* v;
    double idx, idy;  // 1/dx, 1/dy for the non-decision lookups of the moves
    // x0, y0, 1/dx, 1/dy as float pairs (hi + lo) for float-float lookups
    float fx0h, fx0l, fy0h, fy0l, fidxh, fidxl, fidyh, fidyl;
};

// Counters the device accumulates (mesh_stats fields).
struct DevCounters {
    unsigned long long exact_calls, clip_inconsistent, ring_overflow, exact_overflow;
    unsigned long long newton_fail, trace_cap, quad_cap, dup_points;
    // Voronoi work, counted only with debug recording on
    unsigned long long vor_candidates, vor_picks, vor_cuts, vor_rings, vor_wide;
    unsigned long long triangulations;  // iterations that re-triangulated
    unsigned long long vor_fp64, vor_resolve;  // FP64 cut filters, vertices re-solved in double (debug)
    unsigned long long vor_direct;             // cells built from their previous neighbours (debug)
};

// Per-block partial sums written by the emit kernel (a3/a4/a8 and Eq. 3 sums).
struct EmitPartial {
    double n_tri, sqrt_alpha, sqrt_beta, max_alpha, max_beta, min_angle;
    double n_edge, sum_l2, sum_mu2;
    double pad;
};
// Per-block partials of the update kernel.
struct UpdatePartial {
    double size_dev, n_edge;
    double not_small;  // > 0 if some inner point moved at least fac_end*h
    double pad;
};

// Device control block: hybrid state, termination, last statistics.
struct DevCtrl {
    int32_t method_param;   // 0 DM, 1 CVD, 2 hybrid
    int32_t method_now;     // move of the current iteration
    int32_t switched;
    int32_t terminated;
    int32_t iterations;     // executed iterations since the flag was cleared
    int32_t have_prev;
    int32_t small_moves;
    int32_t last_method;
    int32_t ovf_n;          // cells queued for the 32-lane Voronoi pass
    int32_t pad0;
    double prev_a, prev_b, prev_amax;
    double fac_mu;
    double target_min_ang;  // > 0: stop once the minimum angle reaches it
    int32_t target_reached;
    int32_t retri;          // this iteration re-triangulates (DistMesh, Algorithm 1)
    int32_t moved_far;      // some point moved more than fac_retria h_i since the triangulation
    int32_t pad1;
    double n_tri, n_edges, half_a, half_b, max_a, max_b, min_ang, size_dev;
    DevCounters cnt;
};

struct DevParams {
    int32_t bounded, validity, newton_max, trace_max, quad_max_level, debug;
    int32_t adding;     // N_current < N_total: point addition (Sec. 3.6) replaces the switch and termination tests
    int32_t pad_p;
    double fac_F, k_spring, dt, fac_pt, fac_geps, fac_voro_bound, fac_end, T_circ;
    double T_switch, T_end_q, T_end_amax, damping;
    double fac_retria;  // DistMesh re-triangulation threshold factor (0: every iteration)
    double T_add;       // point-addition quality threshold (Sec. 3.6)
    double havg;
    // SDF box (domain box)
    double bx0, by0, bx1, by1;
    // neighbour-bucket grid
    int32_t nbx, nby;
    double bsx, bsy;  // bucket sizes
    // float copies used by the bucket assignment (both kernels use these)
    float bx0f, by0f, ibsxf, ibsyf;
    // float copies for the clipping kernels: box size, bucket sizes, and the
    // bucket-assignment margin 1e-3 max(bsx, bsy)
    float Wf, Hf, bsxf, bsyf, bmargf;
};

// a - b for positions stored as float pairs (hi, lo) with hi + lo = x to 2^-48 |x|;
// relative error below 2^-22 once |a - b| >= 2^-20 (callers fall back to double below)
__device__ __forceinline__ float ff_diff(float ah, float al, float bh, float bl) { return (ah - bh) + (al - bl); }

// (X[j] - xi, Y[j] - yi) formed in double and rounded to float, for points
// closer than ff_diff resolves (|d| < 2^-20): rare, so kept out of line (a
// call that is predicated off issues nothing, while inline code would issue
// its FP64 instructions, predicated off, for every point tested)
template <typename T>
static __device__ __noinline__ float2 close_diff(const T* X, const T* Y, int j, T xi, T yi) {
    return make_float2((float)((double)X[j] - (double)xi), (float)((double)Y[j] - (double)yi));
}

// ---------------------------------------------------------------- fixed FP64 ops
__device__ __forceinline__ double fadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double fsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double fmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return __ddiv_rn(a, b); }

// circumcentre (ox, oy) and circumradius R of triangle (a, b, c), fixed
// formula (the vertex order is part of it: callers pass the canonical order,
// smallest id first, counter-clockwise)
__device__ __forceinline__ void circumcentre_fixed(double ax, double ay, double bx, double by, double cx, double cy,
                                                   double& ox, double& oy, double& R) {
    double bx_ = fsub(bx, ax), by_ = fsub(by, ay), cx_ = fsub(cx, ax), cy_ = fsub(cy, ay);
    double B = fadd(fmul(bx_, bx_), fmul(by_, by_));
    double C = fadd(fmul(cx_, cx_), fmul(cy_, cy_));
    double D = fmul(2.0, fsub(fmul(bx_, cy_), fmul(by_, cx_)));
    double ux = fdiv(fsub(fmul(cy_, B), fmul(by_, C)), D);
    double uy = fdiv(fsub(fmul(bx_, C), fmul(cx_, B)), D);
    ox = fadd(ax, ux);
    oy = fadd(ay, uy);
    R = __dsqrt_rn(fadd(fmul(ux, ux), fmul(uy, uy)));
}

// cell of the grid holding (x, y) and local coordinates, clamped to the grid
__device__ __forceinline__ void grid_locate(const DevGrid& g, double x, double y, int& i, int& j, double& fx,
                                            double& fy) {
    double tx = fdiv(fsub(x, g.x0), g.dx), ty = fdiv(fsub(y, g.y0), g.dy);
    double fi = floor(tx), fj = floor(ty);
    i = !(fi >= 0.0) ? 0 : (fi > (double)(g.nx - 2) ? g.nx - 2 : (int)fi);
    j = !(fj >= 0.0) ? 0 : (fj > (double)(g.ny - 2) ? g.ny - 2 : (int)fj);
    fx = fsub(tx, (double)i);
    fy = fsub(ty, (double)j);
    fx = fx < 0.0 ? 0.0 : (fx > 1.0 ? 1.0 : fx);
    fy = fy < 0.0 ? 0.0 : (fy > 1.0 ? 1.0 : fy);
}

// fixed bilinear interpolation: a = v00 + fx (v10 - v00), b = v01 + fx (v11 - v01), a + fy (b - a)
__device__ __forceinline__ double bilin_fixed(const DevGrid& g, double x, double y) {
    int i, j;
    double fx, fy;
    grid_locate(g, x, y, i, j, fx, fy);
    const float* r0 = g.v + (size_t)j * g.nx + i;
    const float* r1 = r0 + g.nx;
    double v00 = __ldg(r0), v10 = __ldg(r0 + 1), v01 = __ldg(r1), v11 = __ldg(r1 + 1);
    double a = fadd(v00, fmul(fx, fsub(v10, v00)));
    double b = fadd(v01, fmul(fx, fsub(v11, v01)));
    return fadd(a, fmul(fy, fsub(b, a)));
}

// bilinear value and its exact derivatives (f_xx = f_yy = 0), FMAs allowed
template <typename T>
__device__ __forceinline__ void bilin_grad(const DevGrid& g, T x, T y, T& f, T& fx_, T& fy_, T& fxy) {
    T tx = (x - (T)g.x0) * (T)g.idx, ty = (y - (T)g.y0) * (T)g.idy;
    T fi = floor(tx), fj = floor(ty);
    int i = !(fi >= (T)0) ? 0 : (fi > (T)(g.nx - 2) ? g.nx - 2 : (int)fi);
    int j = !(fj >= (T)0) ? 0 : (fj > (T)(g.ny - 2) ? g.ny - 2 : (int)fj);
    T fx = tx - (T)i, fy = ty - (T)j;
    fx = fx < (T)0 ? (T)0 : (fx > (T)1 ? (T)1 : fx);
    fy = fy < (T)0 ? (T)0 : (fy > (T)1 ? (T)1 : fy);
    const float* r0 = g.v + (size_t)j * g.nx + i;
    const float* r1 = r0 + g.nx;
    T v00 = __ldg(r0), v10 = __ldg(r0 + 1), v01 = __ldg(r1), v11 = __ldg(r1 + 1);
    T a = v00 + fx * (v10 - v00);
    T b = v01 + fx * (v11 - v01);
    f = a + fy * (b - a);
    T d0 = v10 - v00, d1 = v11 - v01;
    fx_ = (d0 + fy * (d1 - d0)) * (T)g.idx;
    fy_ = (b - a) * (T)g.idy;
    fxy = (d1 - d0) * ((T)g.idx * (T)g.idy);
}

// bilinear value in precision T (FMAs allowed): used for the moves
template <typename T>
__device__ __forceinline__ T bilin(const DevGrid& g, T x, T y) {
    T tx = (x - (T)g.x0) * (T)g.idx, ty = (y - (T)g.y0) * (T)g.idy;
    T fi = floor(tx), fj = floor(ty);
    int i = !(fi >= (T)0) ? 0 : (fi > (T)(g.nx - 2) ? g.nx - 2 : (int)fi);
    int j = !(fj >= (T)0) ? 0 : (fj > (T)(g.ny - 2) ? g.ny - 2 : (int)fj);
    T fx = tx - (T)i, fy = ty - (T)j;
    fx = fx < (T)0 ? (T)0 : (fx > (T)1 ? (T)1 : fx);
    fy = fy < (T)0 ? (T)0 : (fy > (T)1 ? (T)1 : fy);
    const float* r0 = g.v + (size_t)j * g.nx + i;
    const float* r1 = r0 + g.nx;
    T v00 = __ldg(r0), v10 = __ldg(r0 + 1), v01 = __ldg(r1), v11 = __ldg(r1 + 1);
    T a = v00 + fx * (v10 - v00);
    T b = v01 + fx * (v11 - v01);
    return a + fy * (b - a);
}

// geometry cell of a point by the fixed formula floor((x - x0) / dx); returns
// whether the point lies on the grid; (gi, gj) is clamped either way
__device__ __forceinline__ bool point_cell_fixed(const DevGrid& s, double x, double y, int& gi, int& gj) {
    double tx = fdiv(fsub(x, s.x0), s.dx), ty = fdiv(fsub(y, s.y0), s.dy);
    double fi = floor(tx), fj = floor(ty);
    int ncx = s.nx - 1, ncy = s.ny - 1;
    bool inside = fi >= 0.0 && fi <= (double)(ncx - 1) && fj >= 0.0 && fj <= (double)(ncy - 1);
    gi = !(fi >= 0.0) ? 0 : (fi > (double)(ncx - 1) ? ncx - 1 : (int)fi);
    gj = !(fj >= 0.0) ? 0 : (fj > (double)(ncy - 1) ? ncy - 1 : (int)fj);
    return inside;
}

// same lookup in precision T (approximate near cell edges): used by the moves
template <typename T>
__device__ __forceinline__ bool point_cell_t(const DevGrid& s, T x, T y, int& gi, int& gj) {
    T tx = (x - (T)s.x0) * (T)s.idx, ty = (y - (T)s.y0) * (T)s.idy;
    T fi = floor(tx), fj = floor(ty);
    int ncx = s.nx - 1, ncy = s.ny - 1;
    bool inside = fi >= (T)0 && fi <= (T)(ncx - 1) && fj >= (T)0 && fj <= (T)(ncy - 1);
    gi = !(fi >= (T)0) ? 0 : (fi > (T)(ncx - 1) ? ncx - 1 : (int)fi);
    gj = !(fj >= (T)0) ? 0 : (fj > (T)(ncy - 1) ? ncy - 1 : (int)fj);
    return inside;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace trime
