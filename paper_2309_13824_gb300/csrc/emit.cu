// emit.cu -- a3/a4: Delaunay triangles read off the cells and the valid ones
// kept (TriMe++ Sec. 4.1, Procedure I; duality Sec. 1.1), plus the per-block
// quality sums of a8 (Sec. 3.6 Eqs. 11-12) and the DistMesh sums of Eq. 3.
//
// One thread per cell.  Consecutive bisector edges (j, k) of cell i's ring
// meet at the circumcentre c of the CCW triangle (i, j, k).  The triangle is
// emitted iff c lies in Reg_i, Reg_j and Reg_k (octagon of span S = fac*h
// intersected with the domain box) and is valid iff Tests 1-3 pass; both are
// decided by fixed FP64 formulas evaluated on the canonical order (smallest
// id first, CCW), so the three cells of a triangle always agree.  A float
// evaluation with a proven error bound decides first when it is far from the
// threshold.  Cell i records the result as bit t of vmask[i]; the triangle
// is counted once, by its smallest-id vertex.
#include "ff.cuh"
#include "kernels.cuh"

namespace trime {

constexpr float kEpsF = 5.9604645e-8f;  // 2^-24

// c in Reg_v = Oct_v (span S_v) cap domain box, fixed formula
__device__ __forceinline__ bool reg_contains_fixed(const DevParams& P, double px, double py, double h, double cx,
                                                   double cy) {
    if (!(cx >= P.bx0 && cx <= P.bx1 && cy >= P.by0 && cy <= P.by1)) return false;
    if (!P.bounded) return true;
    double S = fmul(P.fac_voro_bound, h);
    double dx = fsub(cx, px), dy = fsub(cy, py);
    return fabs(dx) <= S && fabs(dy) <= S && fabs(fmul(kRT, fadd(dx, dy))) <= S &&
           fabs(fmul(kRT, fsub(dy, dx))) <= S;
}

struct Tri {
    double x[3], y[3];
    double h[3];
};

// Tests 1-3 on the canonical order (a = smallest id, CCW)
static __device__ __noinline__ bool valid_fixed(const MeshView& V, const Tri& t) {
    const DevGrid& s = V.sdf;
    int ncx = s.nx - 1;
    double gx = fdiv(fadd(fadd(t.x[0], t.x[1]), t.x[2]), 3.0);
    double gy = fdiv(fadd(fadd(t.y[0], t.y[1]), t.y[2]), 3.0);
    int gi, gj;
    if (!point_cell_fixed(s, gx, gy, gi, gj)) return false;
    int c = gj * ncx + gi;
    uint8_t k = V.gcls[c];
    if (k == CELL_INNER) return true;
    if (k == CELL_OUTER) return false;
    if (bilin_fixed(s, gx, gy) > V.ggeps[c]) return false;
    int count = 0;
    for (int e = 0; e < 3; e++) {
        int f = e == 2 ? 0 : e + 1;
        double mx = fmul(fadd(t.x[e], t.x[f]), 0.5), my = fmul(fadd(t.y[e], t.y[f]), 0.5);
        if (!point_cell_fixed(s, mx, my, gi, gj)) continue;
        int q = gj * ncx + gi;
        if (V.gcls[q] == CELL_INNER) count++;
        else if (V.gcls[q] == CELL_BOUNDARY && bilin_fixed(s, mx, my) <= V.ggeps[q]) count++;
    }
    if (count >= 2) return true;
    double ox, oy, R;
    circumcentre_fixed(t.x[0], t.y[0], t.x[1], t.y[1], t.x[2], t.y[2], ox, oy, R);
    return fdiv(fabs(bilin_fixed(s, ox, oy)), R) <= V.P.T_circ;
}

struct Nbr {
    int slot, id, cell;
    float dx, dy;  // relative to the cell's generator
    float S;       // octagon span at the neighbour's geometry cell
};

// per-cell constants shared by all the cell's triangles
struct CellC {
    float S;               // octagon span of the generator
    float lx, hx, ly, hy;  // domain box relative to the generator
    float tx, ty;          // generator's grid coordinates (x - x0) / dx
    float idx, idy;        // 1 / dx, 1 / dy
};

template <typename T>
__device__ __forceinline__ Nbr load_nbr(const IterArgs<T>& a, int lab, float4 pi4, T xi, T yi) {
    Nbr n;
    n.slot = lab;
    if (lab >= 0) {
        float4 pj4 = a.pf[lab];
        n.id = a.srt.id[lab];
        n.cell = a.cell[lab];
        n.dx = ff_diff(pj4.x, pj4.y, pi4.x, pi4.y);
        n.dy = ff_diff(pj4.z, pj4.w, pi4.z, pi4.w);
        if (sizeof(T) == 8 && n.dx * n.dx + n.dy * n.dy < 9.094947e-13f) {  // |d| < 2^-20
            const float2 e = close_diff<T>(a.srt.x, a.srt.y, lab, xi, yi);
            n.dx = e.x;
            n.dy = e.y;
        }
        n.S = a.pS[lab];
    } else {
        n.id = 0;
        n.cell = 0;
        n.dx = n.dy = 0.f;
        n.S = 0.f;
    }
    return n;
}

template <typename T>
static __device__ __noinline__ bool emitted_fixed(const IterArgs<T>& a, const MeshView& V, int idi, int ci, T xi,
                                                  T yi, int js, int jid, int jcell, int ks, int kid, int kcell);

// emission decision for (i, j, k), CCW as seen from cell i
template <typename T>
__device__ bool emitted(const IterArgs<T>& a, const MeshView& V, const CellC& cc, int idi, int ci, T xi, T yi,
                        const Nbr& j, const Nbr& k) {
    const DevParams& P = V.P;
    float ax = j.dx, ay = j.dy, bx = k.dx, by = k.dy;
    float M = ax * by - ay * bx;
    float PM = fabsf(ax * by) + fabsf(ay * bx);
    if (M > 64.0f * kEpsF * PM && PM > 1e-30f) {
        float al = ax * ax + ay * ay, bl = bx * bx + by * by;
        float i2M = 0.5f / M;
        float ux = (al * by - bl * ay) * i2M, uy = (bl * ax - al * bx) * i2M;
        float un = fabsf(ux) + fabsf(uy);
        float eu = 64.0f * kEpsF * ((al * fabsf(by) + bl * fabsf(ay)) + (bl * fabsf(ax) + al * fabsf(bx)) + 2.0f * un * PM) *
                   i2M;
        int state = 1;  // 1 inside, 0 outside, 2 undecided
        float mgb = eu + 4.0f * kEpsF * (un + fabsf(cc.lx) + fabsf(cc.hx) + fabsf(cc.ly) + fabsf(cc.hy)) + 1e-7f;
        float bo = fmaxf(fmaxf(cc.lx - ux, ux - cc.hx), fmaxf(cc.ly - uy, uy - cc.hy));  // > 0 outside
        if (bo > mgb) state = 0;
        else if (bo > -mgb) state = 2;
        if (state != 0 && P.bounded) {
            for (int v = 0; v < 3 && state != 0; v++) {
                float dvx = v == 0 ? 0.f : (v == 1 ? j.dx : k.dx), dvy = v == 0 ? 0.f : (v == 1 ? j.dy : k.dy);
                float S = v == 0 ? cc.S : (v == 1 ? j.S : k.S);
                float wx = ux - dvx, wy = uy - dvy;
                float f = fmaxf(fmaxf(fabsf(wx), fabsf(wy)), 0.70710678f * fmaxf(fabsf(wx + wy), fabsf(wy - wx)));
                float mg = eu + 4.0f * kEpsF * (un + fabsf(dvx) + fabsf(dvy)) + 1e-6f * S;
                if (f > S + mg) state = 0;
                else if (f > S - mg) state = 2;
            }
        }
        if (state != 2) return state == 1;
    }
    return emitted_fixed<T>(a, V, idi, ci, xi, yi, j.slot, j.id, j.cell, k.slot, k.id, k.cell);
}

// the fixed FP64 formula on the canonical order (the float filter above
// leaves about 1e-4 decisions per cell to it: out of line, so that its FP64
// instructions are not issued for every triangle)
template <typename T>
static __device__ __noinline__ bool emitted_fixed(const IterArgs<T>& a, const MeshView& V, int idi, int ci, T xi,
                                                  T yi, int js, int jid, int jcell, int ks, int kid, int kcell) {
    const DevParams& P = V.P;
    double xs[3] = {(double)xi, (double)a.srt.x[js], (double)a.srt.x[ks]};
    double ys[3] = {(double)yi, (double)a.srt.y[js], (double)a.srt.y[ks]};
    int ids[3] = {idi, jid, kid};
    int cells[3] = {ci, jcell, kcell};
    int r = 0;
    if (ids[1] < ids[r]) r = 1;
    if (ids[2] < ids[r]) r = 2;
    int o1 = r == 2 ? 0 : r + 1, o2 = o1 == 2 ? 0 : o1 + 1;
    double ox, oy, R;
    circumcentre_fixed(xs[r], ys[r], xs[o1], ys[o1], xs[o2], ys[o2], ox, oy, R);
    for (int v = 0; v < 3; v++)
        if (!reg_contains_fixed(P, xs[v], ys[v], V.gh[cells[v]], ox, oy)) return false;
    return true;
}

// A grid point located in float: its cell is certain when the grid
// coordinate is more than em (its error bound) away from a cell edge.
struct FLoc {
    int gi, gj;
    float fx, fy, emx, emy;
    bool ok, off;
};

__device__ __forceinline__ FLoc locate_f(float tx, float ty, int ncx, int ncy) {
    FLoc L;
    float fi = floorf(tx), fj = floorf(ty);
    L.fx = tx - fi;
    L.fy = ty - fj;
    L.emx = 2.5e-7f * fabsf(tx) + 1e-4f;
    L.emy = 2.5e-7f * fabsf(ty) + 1e-4f;
    L.ok = L.fx > L.emx && L.fx < 1.0f - L.emx && L.fy > L.emy && L.fy < 1.0f - L.emy;
    L.gi = (int)fi;
    L.gj = (int)fj;
    L.off = L.gi < 0 || L.gj < 0 || L.gi >= ncx || L.gj >= ncy;
    return L;
}

// SDF at a located point vs threshold thr: +1 value certainly above, -1
// certainly at or below, 0 undecided.  The bound covers the coordinate error
// (em times the cell's value differences) and float rounding.
__device__ __forceinline__ int sdf_cmp_f(const DevGrid& g, const FLoc& L, float thr) {
    const float* r0 = g.v + (size_t)L.gj * g.nx + L.gi;
    const float* r1 = r0 + g.nx;
    float v00 = __ldg(r0), v10 = __ldg(r0 + 1), v01 = __ldg(r1), v11 = __ldg(r1 + 1);
    float a = v00 + L.fx * (v10 - v00), b = v01 + L.fx * (v11 - v01);
    float val = a + L.fy * (b - a);
    float err = L.emx * (fabsf(v10 - v00) + fabsf(v11 - v01)) + L.emy * fabsf(b - a) +
                1e-6f * (fabsf(v00) + fabsf(v10) + fabsf(v01) + fabsf(v11)) + 2.4e-7f * fabsf(thr);
    if (val > thr + err) return 1;
    if (val < thr - err) return -1;
    return 0;
}

// Tests 1-2 in float on positions relative to p_i: 1 valid, 0 invalid,
// -1 undecided (the fixed FP64 formulas decide; Test 3 always goes there)
__device__ int valid_float(const MeshView& V, const CellC& cc, const Nbr& j, const Nbr& k) {
    int ncx = V.sdf.nx - 1, ncy = V.sdf.ny - 1;
    float gx = (j.dx + k.dx) * (1.0f / 3.0f), gy = (j.dy + k.dy) * (1.0f / 3.0f);
    FLoc L = locate_f(cc.tx + gx * cc.idx, cc.ty + gy * cc.idy, ncx, ncy);
    if (!L.ok) return -1;
    if (L.off) return 0;
    int c = L.gj * ncx + L.gi;
    uint8_t cls = V.gcls[c];
    if (cls == CELL_INNER) return 1;
    if (cls == CELL_OUTER) return 0;
    int r = sdf_cmp_f(V.sdf, L, (float)V.ggeps[c]);
    if (r == 1) return 0;
    if (r == 0) return -1;
    // Test 2: edge midpoints (0, j)/2, (j + k)/2, (k, 0)/2 relative to p_i
    int count = 0;
    for (int e = 0; e < 3; e++) {
        float mx = e == 0 ? 0.5f * j.dx : (e == 1 ? 0.5f * (j.dx + k.dx) : 0.5f * k.dx);
        float my = e == 0 ? 0.5f * j.dy : (e == 1 ? 0.5f * (j.dy + k.dy) : 0.5f * k.dy);
        FLoc M = locate_f(cc.tx + mx * cc.idx, cc.ty + my * cc.idy, ncx, ncy);
        if (!M.ok) return -1;
        if (M.off) continue;
        int q = M.gj * ncx + M.gi;
        uint8_t qc = V.gcls[q];
        if (qc == CELL_INNER) {
            count++;
        } else if (qc == CELL_BOUNDARY) {
            int rr = sdf_cmp_f(V.sdf, M, (float)V.ggeps[q]);
            if (rr == 0) return -1;
            if (rr == -1) count++;
        }
    }
    if (count >= 2) return 1;
    return -1;
}

template <typename T>
__device__ bool valid_tri(const IterArgs<T>& a, const MeshView& V, const CellC& cc, int idi, int ci, T xi, T yi,
                          const Nbr& j, const Nbr& k) {
    if (!V.P.validity) return true;
    // Test 1 shortcut: every cell within gidist of p_i's cell is inner
    float gx = (j.dx + k.dx) * (1.0f / 3.0f), gy = (j.dy + k.dy) * (1.0f / 3.0f);
    float off = fmaxf(fabsf(gx * cc.idx), fabsf(gy * cc.idy));
    if (off + 2.01f < (float)V.gidist[ci]) return true;
    int f = valid_float(V, cc, j, k);
    if (f >= 0) return f == 1;
    int ids[3] = {idi, j.id, k.id};
    double xs[3] = {(double)xi, (double)a.srt.x[j.slot], (double)a.srt.x[k.slot]};
    double ys[3] = {(double)yi, (double)a.srt.y[j.slot], (double)a.srt.y[k.slot]};
    int r = 0;
    if (ids[1] < ids[r]) r = 1;
    if (ids[2] < ids[r]) r = 2;
    int o1 = r == 2 ? 0 : r + 1, o2 = o1 == 2 ? 0 : o1 + 1;
    Tri t;
    t.x[0] = xs[r]; t.y[0] = ys[r];
    t.x[1] = xs[o1]; t.y[1] = ys[o1];
    t.x[2] = xs[o2]; t.y[2] = ys[o2];
    return valid_fixed(V, t);
}

// one block per chunk of kThreads slots (one mesh in a batch)
template <typename T, bool B>
__global__ void __launch_bounds__(kThreads) k_emit(const __grid_constant__ IterArgs<T> a) {
    const MeshView& V = mesh_of<B>(a, blockIdx.x * kThreads);
    if (skip_rebuild(V.ctrl, a.force)) return;
    const bool cvd_now = V.ctrl->method_param == 1 || (V.ctrl->method_param == 2 && V.ctrl->switched);
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    // per-thread sums: triangle count, sum sqrt(alpha), sum sqrt(beta), max
    // alpha, max beta, min angle; valid-edge count and the Eq. 3 sums
    int nt = 0, nedge = 0;
    float q1 = 0.f, q2 = 0.f, q3 = 0.f, q4 = 0.f, q5 = 180.f;
    ff s7{0.f, 0.f}, s8{0.f, 0.f};
    if (s < a.n && (!B || s - V.soff < V.n)) {
        int ne = a.ring_n[s];
        int lab[kRingCap];
        const int4* row = reinterpret_cast<const int4*>(a.ring + (size_t)s * kRingCap);
        for (int q = 0; q < (ne + 3) / 4; q++) {
            int4 v = row[q];
            lab[4 * q] = v.x;
            lab[4 * q + 1] = v.y;
            lab[4 * q + 2] = v.z;
            lab[4 * q + 3] = v.w;
        }
        T xi = a.srt.x[s], yi = a.srt.y[s];
        int idi = a.srt.id[s];
        int ci = a.cell[s];
        uint64_t vm = 0;
        if (ne >= 2) {
            CellC cc;
            const float4 pi4 = a.pf[s];
            cc.S = a.pS[s];
            double xd = (double)xi, yd = (double)yi;
            cc.lx = (float)(V.P.bx0 - xd);
            cc.hx = (float)(V.P.bx1 - xd);
            cc.ly = (float)(V.P.by0 - yd);
            cc.hy = (float)(V.P.by1 - yd);
            cc.tx = (float)((xd - V.sdf.x0) * V.sdf.idx);
            cc.ty = (float)((yd - V.sdf.y0) * V.sdf.idy);
            cc.idx = (float)V.sdf.idx;
            cc.idy = (float)V.sdf.idy;
            Nbr first = load_nbr(a, lab[0], pi4, xi, yi);
            Nbr cur = first;
            for (int t = 0; t < ne; t++) {
                Nbr nxt = t + 1 < ne ? load_nbr(a, lab[t + 1], pi4, xi, yi) : first;
                if (cur.slot >= 0 && nxt.slot >= 0 && emitted(a, V, cc, idi, ci, xi, yi, cur, nxt) &&
                    valid_tri(a, V, cc, idi, ci, xi, yi, cur, nxt)) {
                    vm |= 1ull << t;
                    if (idi < cur.id && idi < nxt.id) {
                        // quality of the triangle (Eq. 11), float from the relative coordinates
                        float bx = cur.dx, by = cur.dy, cx = nxt.dx, cy = nxt.dy;
                        float la = sqrtf((bx - cx) * (bx - cx) + (by - cy) * (by - cy));
                        float lb = sqrtf(cx * cx + cy * cy), lc = sqrtf(bx * bx + by * by);
                        float A2 = fabsf(bx * cy - by * cx);
                        float alpha = (la * lb * lc * (la + lb + lc)) / (4.0f * A2 * A2);
                        float lmax = fmaxf(la, fmaxf(lb, lc)), lmin = fminf(la, fminf(lb, lc));
                        // the smallest angle is opposite the shortest side
                        float p = la, q = lb;
                        if (lmin == la) { p = lb; q = lc; }
                        else if (lmin == lb) { p = la; q = lc; }
                        float cs = (p * p + q * q - lmin * lmin) / (2.0f * p * q);
                        cs = fminf(1.0f, fmaxf(-1.0f, cs));
                        float beta = lmax / lmin;
                        nt++;
                        q1 += sqrtf(alpha);
                        q2 += sqrtf(beta);
                        q3 = fmaxf(q3, alpha);
                        q4 = fmaxf(q4, beta);
                        q5 = fminf(q5, acosf(cs) * (180.0f / 3.14159265f));
                    }
                }
                cur = nxt;
            }
            // valid edges (Eq. 3 sums), counted by the smaller id; they set the
            // DistMesh rest lengths, so they stay in T precision unless this
            // iteration's move is CVD (then fac_mu only feeds a statistic).  In
            // FP64 mode both sums run in float-float, the edge vectors exact
            // from the three-float positions.
            const ff fxi{pi4.x, pi4.y}, fyi{pi4.z, pi4.w};
            const float2 pi3 = sizeof(T) == 8 ? a.pf3[s] : make_float2(0.f, 0.f);
            for (int t = 0; t < ne; t++) {
                int j = lab[t];
                if (j < 0) continue;
                int tp = t == 0 ? ne - 1 : t - 1;
                if (!((vm >> t) & 1ull) && !((vm >> tp) & 1ull)) continue;
                if (!(idi < a.srt.id[j])) continue;
                nedge++;
                float4 pj4 = a.pf[j];
                if (cvd_now) {
                    float ex = ff_diff(pj4.x, pj4.y, pi4.x, pi4.y), ey = ff_diff(pj4.z, pj4.w, pi4.z, pi4.w);
                    float muf = bilin<float>(V.siz, pi4.x + 0.5f * ex, pi4.z + 0.5f * ey);
                    s7 = ff_add_f(s7, ex * ex + ey * ey);
                    s8 = ff_add_f(s8, muf * muf);
                    continue;
                }
                if (sizeof(T) == 8) {
                    float2 pj3 = a.pf3[j];
                    ff ex = ff_diff3(pj4.x, pj4.y, pj3.x, pi4.x, pi4.y, pi3.x);
                    ff ey = ff_diff3(pj4.z, pj4.w, pj3.y, pi4.z, pi4.w, pi3.y);
                    s7 = ff_add(s7, ff_add(ff_mul(ex, ex), ff_mul(ey, ey)));
                    ff m = bilin_ff(V.siz, ff_scale2(ff_add(fxi, ff{pj4.x, pj4.y}), 0.5f),
                                    ff_scale2(ff_add(fyi, ff{pj4.z, pj4.w}), 0.5f));
                    s8 = ff_add(s8, ff_mul(m, m));
                } else {
                    T xj = a.srt.x[j], yj = a.srt.y[j];
                    T dx = xj - xi, dy = yj - yi;
                    T mu = bilin<T>(V.siz, (xi + xj) * (T)0.5, (yi + yj) * (T)0.5);
                    s7 = ff_add_f(s7, (float)(dx * dx + dy * dy));
                    s8 = ff_add_f(s8, (float)(mu * mu));
                }
            }
        }
        a.vmask[s] = vm;
    }
    // block reduction into one partial: integers and float extrema within the
    // warp, sums in float-float, then double across the warps
    nt = __reduce_add_sync(0xffffffffu, nt);
    nedge = __reduce_add_sync(0xffffffffu, nedge);
    ff w1 = warp_sum_ff(ff{q1, 0.f}), w2 = warp_sum_ff(ff{q2, 0.f});
    s7 = warp_sum_ff(s7);
    s8 = warp_sum_ff(s8);
    q3 = warp_max(q3);
    q4 = warp_max(q4);
    q5 = -warp_max(-q5);
    __shared__ double sh[kThreads / 32][9];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sh[w][0] = (double)nt;
        sh[w][1] = ff_to_d(w1);
        sh[w][2] = ff_to_d(w2);
        sh[w][3] = (double)q3;
        sh[w][4] = (double)q4;
        sh[w][5] = (double)q5;
        sh[w][6] = (double)nedge;
        sh[w][7] = ff_to_d(s7);
        sh[w][8] = ff_to_d(s8);
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        int q = threadIdx.x;
        double v = sh[0][q];
        for (int k = 1; k < kThreads / 32; k++)
            v = (q == 3 || q == 4) ? fmax(v, sh[k][q]) : (q == 5 ? fmin(v, sh[k][q]) : v + sh[k][q]);
        double* out = reinterpret_cast<double*>(&a.ep[blockIdx.x]);
        out[q] = v;
    }
}

template <typename T>
void launch_emit(const IterArgs<T>& a, int nblocks, cudaStream_t st) {
    if (a.Vs) k_emit<T, true><<<nblocks, kThreads, 0, st>>>(a);
    else k_emit<T, false><<<nblocks, kThreads, 0, st>>>(a);
}
template void launch_emit<double>(const IterArgs<double>&, int, cudaStream_t);

// A DistMesh iteration that keeps the last triangulation (Algorithm 1): the
// state this iteration moves is the current one (cur, slot order), and the
// Eq. 3 sums run over the kept valid edges at the current positions; the
// quality entries of the partials stay neutral.  One block per chunk.
template <typename T, bool B>
__global__ void __launch_bounds__(kThreads) k_dm_keep(const __grid_constant__ IterArgs<T> a) {
    const MeshView& V = mesh_of<B>(a, blockIdx.x * kThreads);
    if (V.ctrl->terminated || V.ctrl->retri) return;
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    int nedge = 0;
    ff s7{0.f, 0.f}, s8{0.f, 0.f};
    if (s < a.n && (!B || s - V.soff < V.n)) {
        T xi = a.cur.x[s], yi = a.cur.y[s];
        a.wrk.x[s] = xi;
        a.wrk.y[s] = yi;
        a.wrk.cls[s] = a.cur.cls[s];
        a.wrk.dprev[s] = a.cur.dprev[s];
        int ne = a.ring_n[s];
        uint64_t vm = a.vmask[s];
        int idi = a.srt.id[s];
        // FP64 mode: squared lengths in double, the sizing in float-float
        // (as in the emit kernel, from positions split into float pairs)
        double s7d = 0.0;
        ff fxi{0.f, 0.f}, fyi{0.f, 0.f};
        if (sizeof(T) == 8) {
            fxi = ff_from_d((double)xi);
            fyi = ff_from_d((double)yi);
        }
        for (int t = 0; t < ne; t++) {
            int j = a.ring[(size_t)s * kRingCap + t];
            if (j < 0) continue;
            int tp = t == 0 ? ne - 1 : t - 1;
            if (!((vm >> t) & 1ull) && !((vm >> tp) & 1ull)) continue;
            if (!(idi < a.srt.id[j])) continue;
            T xj = a.cur.x[j], yj = a.cur.y[j];
            T dx = xj - xi, dy = yj - yi;
            nedge++;
            if (sizeof(T) == 8) {
                s7d += (double)(dx * dx + dy * dy);
                ff m = bilin_ff(V.siz, ff_scale2(ff_add(fxi, ff_from_d((double)xj)), 0.5f),
                                ff_scale2(ff_add(fyi, ff_from_d((double)yj)), 0.5f));
                s8 = ff_add(s8, ff_mul(m, m));
            } else {
                T mu = bilin<T>(V.siz, (xi + xj) * (T)0.5, (yi + yj) * (T)0.5);
                s7 = ff_add_f(s7, (float)(dx * dx + dy * dy));
                s8 = ff_add_f(s8, (float)(mu * mu));
            }
        }
        if (sizeof(T) == 8 && s7d != 0.0) s7 = ff_add(s7, ff_from_d(s7d));
    }
    nedge = __reduce_add_sync(0xffffffffu, nedge);
    s7 = warp_sum_ff(s7);
    s8 = warp_sum_ff(s8);
    __shared__ double sh[kThreads / 32][3];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sh[w][0] = (double)nedge;
        sh[w][1] = ff_to_d(s7);
        sh[w][2] = ff_to_d(s8);
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        int q = threadIdx.x;
        double v = q == 5 ? 180.0 : 0.0;
        if (q >= 6 && q < 9)
            for (int k = 0; k < kThreads / 32; k++) v += sh[k][q - 6];
        reinterpret_cast<double*>(&a.ep[blockIdx.x])[q] = v;
    }
}

template <typename T>
void launch_dm_keep(const IterArgs<T>& a, int nblocks, cudaStream_t st) {
    if (a.Vs) k_dm_keep<T, true><<<nblocks, kThreads, 0, st>>>(a);
    else k_dm_keep<T, false><<<nblocks, kThreads, 0, st>>>(a);
}
template void launch_dm_keep<double>(const IterArgs<double>&, int, cudaStream_t);
template void launch_dm_keep<float>(const IterArgs<float>&, int, cudaStream_t);
template void launch_emit<float>(const IterArgs<float>&, int, cudaStream_t);

// ------------------------------------------------------------------ triangle output
// on the slots [s0, s0 + ns) of one mesh; ids are written relative to s0
template <typename T>
__global__ void k_tri_count(const __grid_constant__ IterArgs<T> a, int32_t s0, int32_t ns, int32_t* cnt) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ns) return;
    int s = s0 + r;
    int ne = a.ring_n[s];
    uint64_t vm = a.vmask[s];
    int idi = a.srt.id[s];
    int c = 0;
    for (int t = 0; t < ne; t++) {
        if (!((vm >> t) & 1ull)) continue;
        int j = a.ring[(size_t)s * kRingCap + t], k = a.ring[(size_t)s * kRingCap + (t + 1 == ne ? 0 : t + 1)];
        if (idi < a.srt.id[j] && idi < a.srt.id[k]) c++;
    }
    cnt[r] = c;
}

template <typename T>
__global__ void k_tri_write(const __grid_constant__ IterArgs<T> a, int32_t s0, int32_t ns, const int32_t* off,
                            int32_t* tri) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ns) return;
    int s = s0 + r;
    int ne = a.ring_n[s];
    uint64_t vm = a.vmask[s];
    int idi = a.srt.id[s];
    int o = off[r];
    for (int t = 0; t < ne; t++) {
        if (!((vm >> t) & 1ull)) continue;
        int j = a.ring[(size_t)s * kRingCap + t], k = a.ring[(size_t)s * kRingCap + (t + 1 == ne ? 0 : t + 1)];
        int idj = a.srt.id[j], idk = a.srt.id[k];
        if (idi < idj && idi < idk) {
            tri[3 * (size_t)o] = idi - s0;
            tri[3 * (size_t)o + 1] = idj - s0;
            tri[3 * (size_t)o + 2] = idk - s0;
            o++;
        }
    }
}

// ------------------------------------------------------------------ medial points
// (Sec. 3.3) of every point of a single mesh, from the emitted triangles: the
// Voronoi vertices of a cell are the circumcentres of its triangles (fixed
// formula on the canonical order).  v1: the one farthest from the point; v2:
// the farthest with (c - p) . (v1 - p) <= 0; ties to the smaller ascending
// vertex-id triple.  Written by id: v[4 id ..] = (v1, v2), flags bit 0 / 1.
__device__ __forceinline__ bool triple_before(int a0, int a1, int a2, int b0, int b1, int b2) {
    // both triples ascending
    if (a0 != b0) return a0 < b0;
    if (a1 != b1) return a1 < b1;
    return a2 < b2;
}

__device__ __forceinline__ void sort3(int& a, int& b, int& c) {
    if (a > b) { int t = a; a = b; b = t; }
    if (b > c) { int t = b; b = c; c = t; }
    if (a > b) { int t = a; a = b; b = t; }
}

template <typename T>
__global__ void k_medial(const __grid_constant__ IterArgs<T> a, int32_t ns, double* v, uint8_t* flags) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    int ne = a.ring_n[s];
    uint64_t vm = a.vmask[s];
    int idi = a.srt.id[s];
    double px = (double)a.srt.x[s], py = (double)a.srt.y[s];
    double best[2] = {-1.0, -1.0}, cx[2] = {0, 0}, cy[2] = {0, 0};
    int tb[2][3] = {{0, 0, 0}, {0, 0, 0}};
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1 && best[0] < 0.0) break;
        double ux = fsub(cx[0], px), uy = fsub(cy[0], py);
        for (int t = 0; t < ne; t++) {
            if (!((vm >> t) & 1ull)) continue;
            int j = a.ring[(size_t)s * kRingCap + t], k = a.ring[(size_t)s * kRingCap + (t + 1 == ne ? 0 : t + 1)];
            int idj = a.srt.id[j], idk = a.srt.id[k];
            // canonical order: smallest id first, counter-clockwise
            int o0 = s, o1 = j, o2 = k;
            if (idj < idi && idj < idk) { o0 = j; o1 = k; o2 = s; }
            else if (idk < idi && idk < idj) { o0 = k; o1 = s; o2 = j; }
            double ox, oy, R;
            circumcentre_fixed((double)a.srt.x[o0], (double)a.srt.y[o0], (double)a.srt.x[o1], (double)a.srt.y[o1],
                               (double)a.srt.x[o2], (double)a.srt.y[o2], ox, oy, R);
            double dx = fsub(ox, px), dy = fsub(oy, py);
            if (pass == 1 && !(fadd(fmul(dx, ux), fmul(dy, uy)) <= 0.0)) continue;
            double d = __dsqrt_rn(fadd(fmul(dx, dx), fmul(dy, dy)));
            int q0 = idi, q1 = idj, q2 = idk;
            sort3(q0, q1, q2);
            if (d > best[pass] ||
                (d == best[pass] && triple_before(q0, q1, q2, tb[pass][0], tb[pass][1], tb[pass][2]))) {
                best[pass] = d;
                cx[pass] = ox;
                cy[pass] = oy;
                tb[pass][0] = q0;
                tb[pass][1] = q1;
                tb[pass][2] = q2;
            }
        }
    }
    uint8_t f = 0;
    double* o = v + 4 * (size_t)idi;
    if (best[0] >= 0.0) {
        o[0] = cx[0];
        o[1] = cy[0];
        f |= 1;
    }
    if (best[1] >= 0.0) {
        o[2] = cx[1];
        o[3] = cy[1];
        f |= 2;
    }
    flags[idi] = f;
}

// the medial points of the cells rebuilt by the big-cell pass (rings of up
// to kBigRing edges); a triangle counts when the fixed formulas emit it and
// find it valid, as the emit kernel decides for ordinary cells
template <typename T>
__global__ void k_medial_big(const __grid_constant__ IterArgs<T> a, int32_t n, const int32_t* rings,
                             const int32_t* lens, double* v, uint8_t* flags) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const MeshView& V = a.V;
    int s = a.ovf3_list[i];
    const int32_t* ring = rings + (size_t)i * kBigRing;
    int ne = lens[i];
    int idi = a.srt.id[s];
    double px = (double)a.srt.x[s], py = (double)a.srt.y[s];
    double best[2] = {-1.0, -1.0}, cx[2] = {0, 0}, cy[2] = {0, 0};
    int tb[2][3] = {{0, 0, 0}, {0, 0, 0}};
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1 && best[0] < 0.0) break;
        double ux = fsub(cx[0], px), uy = fsub(cy[0], py);
        for (int t = 0; t < ne; t++) {
            int j = ring[t], k = ring[t + 1 == ne ? 0 : t + 1];
            if (j < 0 || k < 0) continue;
            double xs[3] = {px, (double)a.srt.x[j], (double)a.srt.x[k]};
            double ys[3] = {py, (double)a.srt.y[j], (double)a.srt.y[k]};
            int ids[3] = {idi, a.srt.id[j], a.srt.id[k]};
            int cells[3] = {a.cell[s], a.cell[j], a.cell[k]};
            int r = 0;
            if (ids[1] < ids[r]) r = 1;
            if (ids[2] < ids[r]) r = 2;
            int o1 = r == 2 ? 0 : r + 1, o2 = o1 == 2 ? 0 : o1 + 1;
            double ox, oy, R;
            circumcentre_fixed(xs[r], ys[r], xs[o1], ys[o1], xs[o2], ys[o2], ox, oy, R);
            bool em = true;
            for (int q = 0; q < 3 && em; q++) em = reg_contains_fixed(V.P, xs[q], ys[q], V.gh[cells[q]], ox, oy);
            if (!em) continue;
            if (V.P.validity) {
                Tri tr;
                tr.x[0] = xs[r]; tr.y[0] = ys[r];
                tr.x[1] = xs[o1]; tr.y[1] = ys[o1];
                tr.x[2] = xs[o2]; tr.y[2] = ys[o2];
                if (!valid_fixed(V, tr)) continue;
            }
            double dx = fsub(ox, px), dy = fsub(oy, py);
            if (pass == 1 && !(fadd(fmul(dx, ux), fmul(dy, uy)) <= 0.0)) continue;
            double d = __dsqrt_rn(fadd(fmul(dx, dx), fmul(dy, dy)));
            int q0 = ids[0], q1 = ids[1], q2 = ids[2];
            sort3(q0, q1, q2);
            if (d > best[pass] ||
                (d == best[pass] && triple_before(q0, q1, q2, tb[pass][0], tb[pass][1], tb[pass][2]))) {
                best[pass] = d;
                cx[pass] = ox;
                cy[pass] = oy;
                tb[pass][0] = q0;
                tb[pass][1] = q1;
                tb[pass][2] = q2;
            }
        }
    }
    uint8_t f = 0;
    double* o = v + 4 * (size_t)idi;
    if (best[0] >= 0.0) {
        o[0] = cx[0];
        o[1] = cy[0];
        f |= 1;
    }
    if (best[1] >= 0.0) {
        o[2] = cx[1];
        o[3] = cy[1];
        f |= 2;
    }
    flags[idi] = f;
}

template <typename T>
void launch_medial_big(const IterArgs<T>& a, int32_t n, const int32_t* rings, const int32_t* lens, double* v,
                       uint8_t* flags, cudaStream_t st) {
    if (n > 0) k_medial_big<T><<<(n + 63) / 64, 64, 0, st>>>(a, n, rings, lens, v, flags);
}
template void launch_medial_big<double>(const IterArgs<double>&, int32_t, const int32_t*, const int32_t*, double*,
                                        uint8_t*, cudaStream_t);
template void launch_medial_big<float>(const IterArgs<float>&, int32_t, const int32_t*, const int32_t*, double*,
                                       uint8_t*, cudaStream_t);

template <typename T>
void launch_medial(const IterArgs<T>& a, int32_t ns, double* v, uint8_t* flags, cudaStream_t st) {
    int g = (ns + kThreads - 1) / kThreads;
    if (g > 0) k_medial<T><<<g, kThreads, 0, st>>>(a, ns, v, flags);
}
template void launch_medial<double>(const IterArgs<double>&, int32_t, double*, uint8_t*, cudaStream_t);
template void launch_medial<float>(const IterArgs<float>&, int32_t, double*, uint8_t*, cudaStream_t);

template <typename T>
void launch_tri_count(const IterArgs<T>& a, int32_t s0, int32_t ns, int32_t* cnt, cudaStream_t st) {
    int g = (ns + kThreads - 1) / kThreads;
    if (g > 0) k_tri_count<T><<<g, kThreads, 0, st>>>(a, s0, ns, cnt);
}
template <typename T>
void launch_tri_write(const IterArgs<T>& a, int32_t s0, int32_t ns, const int32_t* off, int32_t* tri,
                      cudaStream_t st) {
    int g = (ns + kThreads - 1) / kThreads;
    if (g > 0) k_tri_write<T><<<g, kThreads, 0, st>>>(a, s0, ns, off, tri);
}
template void launch_tri_count<double>(const IterArgs<double>&, int32_t, int32_t, int32_t*, cudaStream_t);
template void launch_tri_count<float>(const IterArgs<float>&, int32_t, int32_t, int32_t*, cudaStream_t);
template void launch_tri_write<double>(const IterArgs<double>&, int32_t, int32_t, const int32_t*, int32_t*,
                                       cudaStream_t);
template void launch_tri_write<float>(const IterArgs<float>&, int32_t, int32_t, const int32_t*, int32_t*,
                                      cudaStream_t);

}  // namespace trime
