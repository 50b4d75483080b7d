// voronoi.cuh -- a2: bounded Voronoi cell of every point by half-plane
// clipping (TriMe++ Sec. 2.1 Fig. 3, cell-based approach; Sec. 4.1 octagon
// bound of span S = fac_voro_bound * h_i).
//
// A group of G lanes clips one cell: the convex polygon lives in the group,
// one edge per lane: lane t holds edge E_t as a half-plane n.u <= s (u
// relative to the generator) and the vertex V_t = E_t cap E_{t+1}.  The main
// pass uses G = 8 (four cells per warp; final cells have 6-8 edges); a cell
// that would need more than 8 edges at some step is queued and redone with
// G = 16, then G = 32 by the same code, and one that needs more than 32 by a
// serial pass (one thread per cell, up to 64 edges).
//
// The cell is the intersection of the half-planes of all other points, so
// neither the candidates tried nor their order change it.  A cell starts from
// its edges at the last rebuild: when they still bound a convex polygon that
// winds once with every edge of positive length (checked with the exact
// predicate below), that polygon is taken in one step; otherwise the cell
// starts from the octagon and clips by those previous neighbours first.
// Candidates then come from the bucket grid -- the rows of the disk of
// radius 2 Rmax for a directly built cell, ring by ring otherwise -- filtered
// by that security radius (a point farther than twice the largest vertex
// distance cannot cut), staged in shared memory, tested against every vertex
// at once, and only those that cut are applied, nearest first.  A clip
// classifies every vertex in parallel, finds the single run of cut vertices
// with two ballots and rotates the edge list with shuffles.  Every collective
// operation is executed by the whole warp; a group with nothing to do runs it
// as a no-op.
//
// Exactness: a vertex where two bisectors meet is the circumcentre of
// (i, j, k); the candidate l cuts it iff det4(i,j,k,l) > 0 (l inside that
// circle), decided by a float filter with a proven error bound, then an FP64
// filter, then exact expansion arithmetic with symbolic perturbation.  Other
// vertices involve a bounding line; they are tested in float.  The bounding
// octagon and box used here are enlarged by 1/16 of S over the region Reg_i
// that the emission test reads, so those float decisions cannot change which
// Delaunay triangles have their circumcentre inside Reg_i.
#pragma once
#include "exact.cuh"
#include "kernels.cuh"

namespace trime {

constexpr float kEps = 5.9604645e-8f;  // 2^-24
constexpr unsigned kFull = 0xffffffffu;
constexpr int kStageCap = 64;  // staged candidates per group (16 bytes each; one bit each in a 64-bit mask)
// resident blocks per SM the clipping kernels are compiled for (registers:
// 65536 / (kVoroThreads x this)); a build-time tuning knob
#ifndef TRIME_VORO_MINB
#define TRIME_VORO_MINB 5
#endif

template <int G>
struct Grp {
    int gl;    // lane inside the group
    int goff;  // first warp lane of the group
    __device__ unsigned ballot(bool p) const {
        unsigned b = __ballot_sync(kFull, p);
        return G == 32 ? b : (b >> goff) & ((1u << G) - 1u);
    }
    template <typename V>
    __device__ V shfl(V v, int src) const {
        return __shfl_sync(kFull, v, src, G);
    }
    __device__ float max(float v) const {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
        return v;
    }
};

__device__ __forceinline__ bool warp_any(bool p) { return __any_sync(kFull, p); }

struct Lane {
    float nx, ny, s;      // edge half-plane n.u <= s
    int lab;              // >= 0 bisector (neighbour slot) / < 0 bounding line
    float vx, vy, vR;     // vertex with the next edge and an upper bound of |V|
    int nlab;             // next edge's label
    bool bb;              // vertex of two bisectors
    float Qx, Qy, M;      // det4 filter terms of a bisector-bisector vertex
    float PQx, PQy, PM;   // and their absolute-value permanents
};

// The vertex of n1.u <= s1 and n2.u <= s2 solved in double, where every
// product of two float inputs is exact and the vertex carries a few ulps of
// error; its float rounding then decides the later float cut tests like any
// other vertex.  Returns (ux, uy, |u|, error bound), or w = 0 when the lines
// are parallel or the vertex lies beyond RB.
static __device__ __noinline__ float4 resolve_vertex(float nx, float ny, float s, float nx2, float ny2, float s2,
                                                     float RB) {
    const double Dd = (double)nx * (double)ny2 - (double)ny * (double)nx2;
    if (Dd == 0.0) return make_float4(0.f, 0.f, 0.f, 0.f);
    const double uxd = ((double)s * (double)ny2 - (double)s2 * (double)ny) / Dd;
    const double uyd = ((double)s2 * (double)nx - (double)s * (double)nx2) / Dd;
    const double rd = sqrt(uxd * uxd + uyd * uyd);
    if (!(rd < (double)RB)) return make_float4(0.f, 0.f, 0.f, 0.f);
    return make_float4((float)uxd, (float)uyd, (float)rd, (float)rd * (8.0f * kEps) + 1e-30f);
}

// returns true when the vertex had to be solved again in double
__device__ __forceinline__ bool make_vertex(Lane& L, float nx2, float ny2, float s2, int lab2, float RB) {
    float D = L.nx * ny2 - L.ny * nx2;
    float px = L.s * ny2 - s2 * L.ny, py = s2 * L.nx - L.s * nx2;
    // approximate reciprocal and root (a few ulps): the bound err below
    // allows 64 ulps of the vertex and of r
    float iD = __fdividef(1.0f, D);
    float ux = px * iD, uy = py * iD;
    float q = ux * ux + uy * uy;
    float r = q > 0.0f ? q * rsqrtf(q) : 0.0f;
    float perm = fabsf(L.s * ny2) + fabsf(s2 * L.ny) + fabsf(s2 * L.nx) + fabsf(L.s * nx2) +
                 r * (fabsf(L.nx * ny2) + fabsf(L.ny * nx2));
    float err = 64.0f * kEps * perm * fabsf(iD);
    bool ok = (D != 0.0f) && (r + err < RB);  // false for NaN as well
    const bool resolved = !ok;
    if (!ok) {
        // nearly parallel edges (a bisector almost along a bounding line):
        // the float vertex is too uncertain, so solve again in double (out of
        // line: rare)
        const float4 v = resolve_vertex(L.nx, L.ny, L.s, nx2, ny2, s2, RB);
        if (v.w > 0.0f) {
            ux = v.x;
            uy = v.y;
            r = v.z;
            err = v.w;
            ok = r + err < RB;
        }
    }
    L.vR = ok ? r + err : RB;
    L.vx = ok ? ux : 0.0f;
    L.vy = ok ? uy : 0.0f;
    L.nlab = lab2;
    L.bb = L.lab >= 0 && lab2 >= 0;
    if (L.bb) {
        float ax = L.nx, ay = L.ny, bx = nx2, by = ny2;
        float al = ax * ax + ay * ay, bl = bx * bx + by * by;
        L.M = ax * by - ay * bx;
        L.Qx = bl * ay - al * by;
        L.Qy = al * bx - bl * ax;
        L.PM = fabsf(ax * by) + fabsf(ay * bx);
        L.PQx = al * fabsf(by) + bl * fabsf(ay);
        L.PQy = al * fabsf(bx) + bl * fabsf(ax);
    }
    return resolved;
}

// vertex of this lane with the next lane's edge (all lanes participate)
// what the rare exact path needs besides the launch arguments
struct CellCtx {
    DevCtrl* ctrl;
    int si;   // the cell's slot
    int dbg;  // count the FP64 filters and re-solves
};

template <int G>
__device__ __forceinline__ void lane_vertex(Lane& L, int ne, const Grp<G>& g, float RB, bool active,
                                            const CellCtx& ctx) {
    int nxt = g.gl + 1 >= ne ? 0 : g.gl + 1;
    float nx2 = g.shfl(L.nx, nxt), ny2 = g.shfl(L.ny, nxt);
    float s2 = g.shfl(L.s, nxt);
    int lab2 = g.shfl(L.lab, nxt);
    if (active && g.gl < ne && make_vertex(L, nx2, ny2, s2, lab2, RB) && ctx.dbg)
        atomicAdd(&ctx.ctrl->cnt.vor_resolve, 1ull);
}

// exact decision for vertex (j, k) of cell i against candidate l: FP64 filter,
// then expansion arithmetic with symbolic perturbation
template <typename T>
__device__ __noinline__ bool exact_cut(const IterArgs<T>& a, const CellCtx& c, int sj, int sk, int sl) {
    if (c.dbg) atomicAdd(&c.ctrl->cnt.vor_fp64, 1ull);
    const T* X = a.srt.x;
    const T* Y = a.srt.y;
    double pi[2] = {(double)X[c.si], (double)Y[c.si]};
    double pj[2] = {(double)X[sj], (double)Y[sj]};
    double pk[2] = {(double)X[sk], (double)Y[sk]};
    double pl[2] = {(double)X[sl], (double)Y[sl]};
    double ax = pj[0] - pi[0], ay = pj[1] - pi[1];
    double bx = pk[0] - pi[0], by = pk[1] - pi[1];
    double cx = pl[0] - pi[0], cy = pl[1] - pi[1];
    double al = ax * ax + ay * ay, bl = bx * bx + by * by, cl = cx * cx + cy * cy;
    double lam = al * (bx * cy - by * cx) - bl * (ax * cy - ay * cx) + cl * (ax * by - ay * bx);
    double P = al * (fabs(bx * cy) + fabs(by * cx)) + bl * (fabs(ax * cy) + fabs(ay * cx)) +
               cl * (fabs(ax * by) + fabs(ay * bx));
    if (P > 1e-280 && fabs(lam) > 64.0 * 1.1102230246251565e-16 * P) return lam < 0.0;  // lam = -det4
    atomicAdd(&c.ctrl->cnt.exact_calls, 1ull);
    int o = orient_exact(pi, pj, pk);
    const int32_t* id = a.srt.id;
    int d = incircle_sos(pi, id[c.si], pj, id[sj], pk, id[sk], pl, id[sl]);
    if (o == kExactFail || d == kExactFail) {
        atomicAdd(&c.ctrl->cnt.exact_overflow, 1ull);
        return false;
    }
    return d * o > 0;
}

// Does the half-plane n.u <= s (label lab; bisector: a neighbour's bisector,
// n = d, s = |d|^2/2) cut this lane's vertex?  A vertex on the candidate's
// own line (the candidate already is one of its two edges) is not cut.
template <typename T>
__device__ __forceinline__ bool cuts(const Lane& L, float nx, float ny, float s, int lab, bool bisector,
                                     const IterArgs<T>& a, const CellCtx& ctx) {
    if (lab == L.lab || lab == L.nlab) return false;
    if (bisector && L.bb) {
        float cl = 2.0f * s;
        float lam = fmaf(nx, L.Qx, fmaf(ny, L.Qy, cl * L.M));
        float P = fabsf(nx) * L.PQx + fabsf(ny) * L.PQy + cl * L.PM;
        float bound = 32.0f * kEps * P;
        if (P > 1e-30f && lam < -bound) return true;
        if (P > 1e-30f && lam > bound) return false;
        return exact_cut<T>(a, ctx, L.lab, L.nlab, lab);
    }
    return nx * L.vx + ny * L.vy > s;
}

// Clip the group's polygon by n.u <= s (label lab) when `active`; bisector:
// a neighbour's bisector (n = d, s = |d|^2/2).  Executed by every lane of the
// warp.  Returns 0 ok / no-op, 1 empty cell, 2 more than G edges; any_cut
// tells whether some cell of the warp changed.
template <typename T, int G>
__device__ int clip_by(Lane& L, int& ne, float nx, float ny, float s, int lab, bool bisector, bool active, float RB,
                       const Grp<G>& g, const IterArgs<T>& a, const CellCtx& ctx, bool& any_cut) {
    bool cut = active && g.gl < ne && cuts<T>(L, nx, ny, s, lab, bisector, a, ctx);
    unsigned m = g.ballot(cut);
    unsigned full = ne >= 32 ? kFull : ((1u << ne) - 1u);
    int status = 0;
    bool doit = active && m != 0;
    if (doit && (m & full) == full) {
        status = 1;
        doit = false;
    }
    any_cut = warp_any(doit);
    if (!any_cut) return status;  // nothing to cut anywhere in the warp
    int prevl = g.gl == 0 ? ne - 1 : g.gl - 1;
    bool pcut = (m >> (prevl & 31)) & 1u;
    unsigned starts = g.ballot(g.gl < ne && cut && !pcut);
    unsigned ends = g.ballot(g.gl < ne && !cut && pcut);
    if (doit && __popc(starts) != 1 && g.gl == 0) atomicAdd(&ctx.ctrl->cnt.clip_inconsistent, 1ull);
    int sidx = starts ? __ffs(starts) - 1 : 0;
    unsigned after = sidx >= 31 ? 0u : (ends >> (sidx + 1)) << (sidx + 1);
    int eidx = after ? __ffs(after) - 1 : (ends ? __ffs(ends) - 1 : 0);
    int k = sidx - eidx + 1;  // kept edges E_e .. E_s
    if (k <= 0) k += ne;
    int nn = k + 1;
    if (doit && nn > G) {
        status = 2;
        doit = false;
    }
    // rotate the edges so E_e lands in lane 0, append the new edge in lane k,
    // then every lane recomputes its vertex (SIMT: as cheap as two lanes)
    int src = eidx + g.gl;  // (eidx + gl) mod ne for the lanes that keep an edge
    if (src >= ne) src -= ne;
    if (!doit) src = g.gl;
    float rnx = g.shfl(L.nx, src), rny = g.shfl(L.ny, src), rs = g.shfl(L.s, src);
    int rlab = g.shfl(L.lab, src);
    if (doit) {
        if (g.gl < k) {
            L.nx = rnx;
            L.ny = rny;
            L.s = rs;
            L.lab = rlab;
        } else if (g.gl == k) {
            L.nx = nx;
            L.ny = ny;
            L.s = s;
            L.lab = lab;
        }
        ne = nn;
    }
    lane_vertex<G>(L, ne, g, RB, doit, ctx);
    return status;
}

// monotone key of a direction's angle, in [0, 4): the quadrant (decided by
// the signs) plus a fraction that grows with the angle inside it
__device__ __forceinline__ float dir_key(float x, float y) {
    if (y >= 0.0f && x > 0.0f) return __fdividef(y, x + y);
    if (x <= 0.0f && y > 0.0f) return 1.0f + __fdividef(-x, y - x);
    if (y <= 0.0f && x < 0.0f) return 2.0f + __fdividef(-y, -x - y);
    return 3.0f + __fdividef(x, x - y);
}

// the half-plane n.u <= s of a bounding-plane label, relative to the
// generator: octagon plane k (label -1 - k) with normal (cos k pi/4,
// sin k pi/4) at the span SB; domain-box plane b (label -9 - b: left, right,
// bottom, top) enlarged by mb; (xf, yf) the generator relative to the box's
// lower corner, W x H the box
__device__ __forceinline__ void bounding_plane(int lab, float SB, float xf, float yf, float W, float H, float mb,
                                               float& nx, float& ny, float& s) {
    constexpr float h = 0.70710678f;
    if (lab >= oct_label(7)) {
        const int k = -1 - lab;
        const int c = (k + 6) & 7;
        nx = k == 0 ? 1.f : k == 4 ? -1.f : (k == 2 || k == 6) ? 0.f : (k == 1 || k == 7) ? h : -h;
        ny = c == 0 ? 1.f : c == 4 ? -1.f : (c == 2 || c == 6) ? 0.f : (c == 1 || c == 7) ? h : -h;
        s = SB;
    } else {
        const int b = -9 - lab;
        nx = b == 0 ? -1.f : (b == 1 ? 1.f : 0.f);
        ny = b == 2 ? -1.f : (b == 3 ? 1.f : 0.f);
        s = b == 0 ? xf + mb : b == 1 ? (W - xf) + mb : b == 2 ? yf + mb : (H - yf) + mb;
    }
}

// one cell per group; slot < 0 marks an idle group (it still takes part in
// every collective operation of its warp).  DISK: directly built cells read
// their security disk's bucket rows in one pass; without it (the batched
// kernels, whose register budget the second reading loop would strain) every
// cell reads bucket rings.
template <typename T, int G, bool DISK>
__device__ void voronoi_cell(const IterArgs<T>& a, const MeshView& V, int slot, const Grp<G>& g, float4* stage) {
    const DevParams& P = V.P;
    const float INF = __int_as_float(0x7f800000);
    bool live = slot >= 0;
    int s = live ? slot : 0;
    if (live && a.dom[s]) {
        if (g.gl == 0) {
            a.ring_n[s] = 0;
            a.cellR[s] = 0.0f;
        }
        live = false;
    }
    const float4 pi4 = a.pf[s];
    CellCtx ctx;
    ctx.ctrl = V.ctrl;
    ctx.si = s;
    ctx.dbg = P.debug;
    // generator relative to the box corner, and the box size (float; the box
    // planes only need to bound Reg_i with the S/16 margin)
    const float xf = (pi4.x - P.bx0f) + pi4.y, yf = (pi4.z - P.by0f) + pi4.w;
    const float Wf = P.Wf, Hf = P.Hf;
    float RB, mb, SB = 0.0f;
    if (P.bounded) {
        float S = a.pS[s];
        SB = S * (17.0f / 16.0f);
        RB = SB * 1.0824459f * 1.0001f;  // octagon circumradius SB / cos(pi/8)
        mb = S * (1.0f / 16.0f);
    } else {
        mb = 0.125f * (Wf > Hf ? Wf : Hf);
        RB = (sqrtf(Wf * Wf + Hf * Hf) + 4.0f * mb) * 1.0001f;
    }
    Lane L;
    L.nx = L.ny = L.s = 0.0f;
    L.lab = -1;
    L.bb = false;
    L.vR = 0.0f;
    L.vx = L.vy = 0.0f;
    L.nlab = -1;
    L.M = L.Qx = L.Qy = L.PM = L.PQx = L.PQy = 0.0f;
    int ne = 0;
    int status = 0;

    // the cell's edges at the last rebuild, one per lane in ring order
    // (points move little between rebuilds): a neighbour's slot, a
    // bounding-plane label or an empty entry.  (wdx, wdy, ws): the edge's
    // half-plane n.u <= s; wd2 = |d|^2 for a neighbour.
    int wl = kNoLabel;
    if (live && g.gl < kWarm) wl = a.warm[(size_t)s * kWarm + g.gl];
    const bool wbis = wl >= 0 && wl != s;
    bool wvalid = false;
    float wdx = 0.f, wdy = 0.f, wd2 = INF, ws = 0.f;
    if (wbis) {
        float4 pj4 = a.pf[wl];
        wdx = ff_diff(pj4.x, pj4.y, pi4.x, pi4.y);
        wdy = ff_diff(pj4.z, pj4.w, pi4.z, pi4.w);
        wd2 = wdx * wdx + wdy * wdy;
        if (sizeof(T) == 8 && wd2 < 9.094947e-13f) {  // |d| < 2^-20: exact double difference
            const float2 e = close_diff<T>(a.srt.x, a.srt.y, wl, a.srt.x[s], a.srt.y[s]);
            wdx = e.x;
            wdy = e.y;
            wd2 = wdx * wdx + wdy * wdy;
        }
        ws = 0.5f * wd2;
        wvalid = !a.dom[wl] && wd2 > 0.0f;
    } else if (P.bounded && wl < 0 && wl >= box_label(3)) {
        bounding_plane(wl, SB, xf, yf, Wf, Hf, mb, wdx, wdy, ws);
        wvalid = true;
    }

    // 1. Direct construction.  If the previous edges, in ring order, each
    // turn left by less than pi (a float filter on the orientation of
    // consecutive normals), wind once around the generator, and every edge
    // keeps a positive length (the vertex of edges t, t+1 strictly inside
    // edge t+2: the exact cut predicate for two bisectors), they bound a
    // convex polygon that is exactly the intersection of their half-planes,
    // built in one step.  An edge without a positive length (a neighbour
    // lost by a flip) is dropped and the rest certified again; a dropped
    // point is tested again with the bucket candidates below, like any other
    // point.  Any other case starts from the octagon (2.).
    const unsigned wm = g.ballot(wvalid);
    const int nw = __popc(wm);
    bool direct = live && P.bounded && nw >= 3 && (wm & (wm + 1u)) == 0u;  // a prefix of the lanes
    if (warp_any(direct)) {
        if (direct) {
            L.nx = wdx;
            L.ny = wdy;
            L.s = ws;
            L.lab = wl;
            ne = nw;
        }
        bool built = false;
#pragma unroll 1
        for (int round = 0; round < 3 && warp_any(direct && !built); round++) {
            const bool act = direct && !built;
            const int n1 = g.gl + 1 >= ne ? 0 : g.gl + 1;
            const int n2 = g.gl + 2 >= ne ? ((g.gl + 2 - ne) & (G - 1)) : g.gl + 2;
            const float key = dir_key(L.nx, L.ny);
            const float ax = g.shfl(L.nx, n1), ay = g.shfl(L.ny, n1), key1 = g.shfl(key, n1);
            const float bx = g.shfl(L.nx, n2), by = g.shfl(L.ny, n2), bs = g.shfl(L.s, n2);
            const int blab = g.shfl(L.lab, n2);
            lane_vertex<G>(L, ne, g, RB, act, ctx);
            bool bad = false, desc = false, flat = false;
            if (act && g.gl < ne) {
                const float D = L.nx * ay - L.ny * ax;
                const float PD = fabsf(L.nx * ay) + fabsf(L.ny * ax);
                desc = key1 < key;
                bad = !(D > 64.0f * kEps * PD) || !(L.vR < RB);
                if (!bad && blab >= 0 && L.bb) {
                    flat = cuts<T>(L, bx, by, bs, blab, true, a, ctx);  // edge t+1 has no length (exact)
                } else if (!bad) {
                    // a bounding plane takes part: a float decision that must
                    // clear the vertex's error bound (vR - |V|) and the
                    // rounding of the dot product; an uncertain case starts
                    // from the octagon
                    const float dot = bx * L.vx + by * L.vy;
                    const float ev = fmaxf(L.vR - sqrtf(L.vx * L.vx + L.vy * L.vy), 0.0f);
                    const float mg = sqrtf(bx * bx + by * by) * ev * 1.01f +
                                     8.0f * kEps * (fabsf(bx * L.vx) + fabsf(by * L.vy) + fabsf(bs));
                    if (dot > bs + mg) flat = true;
                    else if (!(dot < bs - mg)) bad = true;
                }
            }
            const unsigned badm = g.ballot(bad), descm = g.ballot(desc), flatm = g.ballot(flat);
            if (act && (badm != 0u || __popc(descm) != 1)) direct = false;
            else if (act && flatm == 0u) built = true;
            // drop the flagged edges: lane r takes the r-th kept one
            const bool drop = act && direct && !built;
            const unsigned all = (1u << (ne & 31)) - 1u;
            const unsigned rm = drop ? (((flatm << 1) | (flatm >> ((ne - 1) & 31))) & all) : 0u;
            const unsigned keepm = all & ~rm;
            const int nk = __popc(keepm);
            if (drop && nk < 3) direct = false;
            int src = g.gl;
            if (drop && nk >= 3 && g.gl < nk) {
                unsigned mm = keepm;
                for (int q = 0; q < g.gl; q++) mm &= mm - 1u;
                src = __ffs(mm) - 1;
            }
            const float cnx = g.shfl(L.nx, src), cny = g.shfl(L.ny, src), csv = g.shfl(L.s, src);
            const int clab = g.shfl(L.lab, src);
            if (drop && nk >= 3) {
                L.nx = cnx;
                L.ny = cny;
                L.s = csv;
                L.lab = clab;
                ne = nk;
            }
        }
        direct = direct && built;
    }
    if (P.debug && direct && g.gl == 0) atomicAdd(&V.ctrl->cnt.vor_direct, 1ull);
    // 2. Sequential start: the octagon (or the enlarged box)
    const bool seq = live && !direct;
    if (warp_any(seq)) {
        if (seq) {
            ne = P.bounded ? 8 : 4;
            if (P.bounded) {
                // octagon, CCW from the +x normal
                bounding_plane(oct_label(g.gl & 7), SB, xf, yf, Wf, Hf, mb, L.nx, L.ny, L.s);
                L.lab = oct_label(g.gl & 7);
            } else {
                // enlarged box, CCW: bottom, right, top, left
                const int b = g.gl & 3;
                const int bs = b == 0 ? 2 : (b == 1 ? 1 : (b == 2 ? 3 : 0));
                bounding_plane(box_label(bs), SB, xf, yf, Wf, Hf, mb, L.nx, L.ny, L.s);
                L.lab = box_label(bs);
            }
        }
        lane_vertex<G>(L, ne, g, RB, seq, ctx);
    }
    if (P.bounded) {
        // the planes of the octagon (bit k) and of the domain box (bit 8 + b)
        // that cut some vertex: a direct polygon reaching beyond the
        // octagon's inradius, or any polygon when a box plane comes closer
        // than the octagon's circumradius.  The polygon only shrinks, so a
        // plane that cuts none of the vertices never will.
        const bool near_box = live && !(RB * 1.001f < xf + mb && RB * 1.001f < (Wf - xf) + mb &&
                                        RB * 1.001f < yf + mb && RB * 1.001f < (Hf - yf) + mb);
        unsigned pm = 0u;
        if (live && g.gl < ne) {
            if (direct && L.vR > SB) {
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    float nx, ny, sp;
                    bounding_plane(oct_label(k), SB, xf, yf, Wf, Hf, mb, nx, ny, sp);
                    if (cuts<T>(L, nx, ny, sp, oct_label(k), false, a, ctx)) pm |= 1u << k;
                }
            }
            if (near_box) {
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    float nx, ny, sp;
                    bounding_plane(box_label(b), SB, xf, yf, Wf, Hf, mb, nx, ny, sp);
                    if (cuts<T>(L, nx, ny, sp, box_label(b), false, a, ctx)) pm |= 1u << (8 + b);
                }
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) pm |= __shfl_xor_sync(kFull, pm, o);
        unsigned todo = __reduce_or_sync(kFull, pm);
        while (todo) {
            const int k = __ffs(todo) - 1;
            todo &= todo - 1u;
            const int lab = k < 8 ? oct_label(k) : box_label(k - 8);
            float nx, ny, sp;
            bounding_plane(lab, SB, xf, yf, Wf, Hf, mb, nx, ny, sp);
            bool any_cut;
            int st = clip_by<T, G>(L, ne, nx, ny, sp, lab, false, live && status == 0 && ((pm >> k) & 1u), RB, g, a,
                                   ctx, any_cut);
            if (st) status = st;
        }
    }
    float Rmax = g.max(g.gl < ne ? L.vR : 0.0f);
    int bxi, byi;
    bucket_of(P, pi4.x, pi4.z, bxi, byi);
    const float bsx = P.bsxf, bsy = P.bsyf;
    const float bmargin = P.bmargf + 4e-6f * (1.0f + fabsf(xf) + fabsf(yf));
    bool done = !live || status != 0;
    int nst = 0;
    unsigned used = 0;  // per lane: its staged entries (gl, gl + G, ...) already taken or dropped
    // apply the staged entries that are not yet used, nearest first
    // (warp-uniform loop).  The nearest entry is found by a minimum over keys
    // made of the squared distance's bits with the entry index in the lowest
    // 7 (the order of nearly equal distances does not matter for the result).
    auto flush = [&]() {
        while (true) {
            unsigned key = 0xFFFFFFFFu;
            int kq = 0;
            for (int q = g.gl; q < nst; q += G, kq++)
                if (!((used >> kq) & 1u)) key = min(key, (__float_as_uint(stage[q].z) & ~0x7Fu) | (unsigned)q);
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) key = min(key, __shfl_xor_sync(kFull, key, o));
            float lim = 4.0f * Rmax * Rmax * 1.0001f;
            int bi = (int)(key & 0x7Fu);
            bool has = !done && key != 0xFFFFFFFFu && __uint_as_float(key & ~0x7Fu) < lim;
            if (!warp_any(has)) break;
            float4 c = has ? stage[bi] : make_float4(0.f, 0.f, 1.f, 0.f);
            if (has && (bi & (G - 1)) == g.gl) used |= 1u << (bi / G);
            int ne0 = ne;
            bool any_cut;
            int st = clip_by<T, G>(L, ne, c.x, c.y, 0.5f * c.z, __float_as_int(c.w), true, has, RB, g, a, ctx, any_cut);
            if (P.debug && has && g.gl == 0) {
                atomicAdd(&V.ctrl->cnt.vor_picks, 1ull);
                if (ne != ne0 || st) atomicAdd(&V.ctrl->cnt.vor_cuts, 1ull);
            }
            if (st) {
                status = st;
                done = true;
                nst = 0;
            }
            if (any_cut) Rmax = g.max(g.gl < ne ? L.vR : 0.0f);
        }
        nst = 0;
        used = 0;
        __syncwarp();
    };
    // test every staged entry against the polygon at once: an entry that
    // cuts no vertex never will (the polygon only shrinks) and is dropped;
    // the others are applied one by one (flush)
    auto settle = [&]() {
        unsigned long long cm = 0ull;
        if (!done && g.gl < ne) {
            for (int q = 0; q < nst; q++) {
                const float4 c = stage[q];
                if (cuts<T>(L, c.x, c.y, 0.5f * c.z, __float_as_int(c.w), true, a, ctx)) cm |= 1ull << q;
            }
        }
        unsigned lo = (unsigned)cm, hi = (unsigned)(cm >> 32);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            lo |= __shfl_xor_sync(kFull, lo, o);
            hi |= __shfl_xor_sync(kFull, hi, o);
        }
        cm = ((unsigned long long)hi << 32) | lo;
        int kq = 0;
        for (int q = g.gl; q < nst; q += G, kq++)
            if (!((cm >> q) & 1ull)) used |= 1u << kq;
        if (warp_any(cm != 0ull)) flush();
        nst = 0;
        used = 0;
        __syncwarp();
    };
    // sequentially started cells apply their previous neighbours first
    {
        const bool keep = seq && !done && wbis && wvalid && wd2 < 4.0f * Rmax * Rmax * 1.0001f;
        const unsigned km = g.ballot(keep);
        if (keep) stage[__popc(km & ((1u << g.gl) - 1u))] = make_float4(wdx, wdy, wd2, __int_as_float(wl));
        nst = __popc(km);
        __syncwarp();
        if (warp_any(nst > 0)) flush();
    }
    // the slot ranges [lo, hi) of the group's lanes: their points loaded two
    // per lane and step, staged when within 2 Rmax
    auto load = [&](int lo, int hi) {
        int cnt = hi - lo;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            int y = __shfl_up_sync(kFull, incl, o, G);
            if (g.gl >= o) incl += y;
        }
        int total = g.shfl(incl, G - 1);
        int excl = incl - cnt;
        // two candidates per lane and iteration (entries q0 + gl and
        // q0 + G + gl), their loads issued together
        for (int q0 = 0; warp_any(q0 < total); q0 += 2 * G) {
            int cs[2];
            bool valid[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int q = q0 + h * G + g.gl;
                int ow = 0;
#pragma unroll
                for (int step = G / 2; step > 0; step >>= 1) {
                    int pr = ow + step;
                    int ex = g.shfl(excl, pr);
                    if (ex <= q) ow = pr;
                }
                const int olo = g.shfl(lo, ow);
                const int oex = g.shfl(excl, ow);
                cs[h] = olo + (q - oex);
                valid[h] = !done && q < total && cs[h] != s;
            }
            float4 pj4[2];
            bool dup[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                pj4[h] = valid[h] ? a.pf[cs[h]] : make_float4(0.f, 0.f, 0.f, 0.f);
                dup[h] = valid[h] && a.dom[cs[h]];
            }
            float dx[2], dy[2], d2[2];
            bool keep[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                dx[h] = ff_diff(pj4[h].x, pj4[h].y, pi4.x, pi4.y);
                dy[h] = ff_diff(pj4[h].z, pj4[h].w, pi4.z, pi4.w);
                d2[h] = dx[h] * dx[h] + dy[h] * dy[h];
                if (sizeof(T) == 8 && valid[h] && d2[h] < 9.094947e-13f) {  // |d| < 2^-20: exact double difference
                    const float2 e = close_diff<T>(a.srt.x, a.srt.y, cs[h], a.srt.x[s], a.srt.y[s]);
                    dx[h] = e.x;
                    dy[h] = e.y;
                    d2[h] = dx[h] * dx[h] + dy[h] * dy[h];
                }
                keep[h] = valid[h] && !dup[h] && d2[h] < 4.0f * Rmax * Rmax * 1.0001f;
            }
            unsigned km0 = g.ballot(keep[0]), km1 = g.ballot(keep[1]);
            if (warp_any(nst + __popc(km0) + __popc(km1) > kStageCap)) {
                settle();
#pragma unroll
                for (int h = 0; h < 2; h++) keep[h] = keep[h] && !done && d2[h] < 4.0f * Rmax * Rmax * 1.0001f;
                km0 = g.ballot(keep[0]);
                km1 = g.ballot(keep[1]);
            }
            const unsigned lt = (1u << g.gl) - 1u;
            if (keep[0]) stage[nst + __popc(km0 & lt)] = make_float4(dx[0], dy[0], d2[0], __int_as_float(cs[0]));
            if (keep[1])
                stage[nst + __popc(km0) + __popc(km1 & lt)] = make_float4(dx[1], dy[1], d2[1], __int_as_float(cs[1]));
            if (P.debug && g.gl == 0 && (km0 | km1))
                atomicAdd(&V.ctrl->cnt.vor_candidates, (unsigned long long)(__popc(km0) + __popc(km1)));
            nst += __popc(km0) + __popc(km1);
            __syncwarp();
        }
    };
    // a bucket row's column range [c0, c1] trimmed to the chord of the disk
    // of radius 2 Rmax (with the bucket-assignment margin); false when the
    // row holds no point that can cut
    auto trim = [&](int row, int& c0, int& c1) -> bool {
        c0 = c0 < 0 ? 0 : c0;
        c1 = c1 >= P.nbx ? P.nbx - 1 : c1;
        if (row < 0 || row >= P.nby || c0 > c1) return false;
        const float lim = 2.0f * Rmax * 1.0001f + bmargin;
        const float ddy = fmaxf(fmaxf((float)row * bsy - yf, yf - (float)(row + 1) * bsy), 0.0f);
        if (ddy > lim) return false;
        const float w = sqrtf(lim * lim - ddy * ddy) + bmargin;
        c0 = max(c0, (int)floorf((xf - w) / bsx));
        c1 = min(c1, (int)floorf((xf + w) / bsx));
        return c0 <= c1;
    };
    // (1) cells started from the octagon: bucket rings around their own
    // bucket (the 3x3 block, then rings of width 1), each followed by the
    // batched test, until nothing beyond the rings read can cut: their
    // radius shrinks ring by ring
    {
        bool rdone = done || (DISK && !seq);
        for (int r = 1; warp_any(!rdone); r++) {
            if (P.debug && !rdone && g.gl == 0) atomicAdd(&V.ctrl->cnt.vor_rings, 1ull);
            const int nr = r == 1 ? 3 : 4 * r;
            for (int kb = 0; kb < nr; kb += G) {
                const int k = kb + g.gl;
                int lo = 0, hi = 0;
                if (!rdone && k < nr) {
                    int row, c0, c1;
                    if (r == 1) {
                        row = byi - 1 + k;
                        c0 = bxi - 1;
                        c1 = bxi + 1;
                    } else if (k < 2) {
                        row = k == 0 ? byi - r : byi + r;
                        c0 = bxi - r;
                        c1 = bxi + r;
                    } else {
                        const int kk = k - 2;
                        row = byi - r + 1 + (kk >> 1);
                        c0 = c1 = (kk & 1) ? bxi + r : bxi - r;
                    }
                    if (trim(row, c0, c1)) {
                        lo = a.bstart[V.boff + row * P.nbx + c0];
                        hi = a.bstart[V.boff + row * P.nbx + c1 + 1];
                    }
                }
                load(lo, hi);
            }
            settle();
            // nothing outside the (2r+1)^2 block can cut once it is beyond 2 Rmax
            if (!rdone) {
                float dmin = INF;
                if (bxi - r > 0) dmin = fminf(dmin, xf - (float)(bxi - r) * bsx);
                if (bxi + r < P.nbx - 1) dmin = fminf(dmin, (float)(bxi + r + 1) * bsx - xf);
                if (byi - r > 0) dmin = fminf(dmin, yf - (float)(byi - r) * bsy);
                if (byi + r < P.nby - 1) dmin = fminf(dmin, (float)(byi + r + 1) * bsy - yf);
                const bool all = bxi - r <= 0 && bxi + r >= P.nbx - 1 && byi - r <= 0 && byi + r >= P.nby - 1;
                if (done || all || 2.0f * Rmax * 1.0001f < dmin - bmargin) rdone = true;
            }
        }
        if (seq || !DISK) done = true;
    }
    // (2) directly built cells (their radius is close to final): every
    // bucket row that the disk of radius 2 Rmax around the generator
    // reaches, one row per lane from the generator's row outward,
    // each trimmed to the disk's chord with the radius of the moment.  The
    // radius only shrinks, so this one pass holds every point that can cut
    // the cell.
    if constexpr (DISK) {
        if (P.debug && !done && g.gl == 0) atomicAdd(&V.ctrl->cnt.vor_rings, 1ull);
        const float lim = 2.0f * Rmax * 1.0001f + bmargin;
        int rlo = 0, rhi = -1;
        if (!done) {
            rlo = max(0, (int)floorf((yf - lim) / bsy));
            rhi = min(P.nby - 1, (int)floorf((yf + lim) / bsy));
        }
        const int nrows = rhi - rlo + 1;
        const int c = min(max(byi, rlo), max(rhi, rlo));  // the generator's row
        const int na = c - rlo, nb = rhi - c, m = min(na, nb);
        for (int kb = 0; warp_any(kb < nrows); kb += G) {
            const int k = kb + g.gl;
            int lo = 0, hi = 0;
            if (!done && k < nrows) {
                // c, c - 1, c + 1, c - 2, ..., then the longer side's rest
                const int row = k == 0 ? c
                                : k <= 2 * m ? ((k & 1) ? c - (k + 1) / 2 : c + k / 2)
                                             : (na > nb ? c - (k - m) : c + (k - m));
                int c0 = 0, c1 = P.nbx - 1;
                if (trim(row, c0, c1)) {
                    lo = a.bstart[V.boff + row * P.nbx + c0];
                    hi = a.bstart[V.boff + row * P.nbx + c1 + 1];
                }
            }
            load(lo, hi);
        }
        settle();
        done = true;
    }
    // the ring is written from its smallest label on, so that it depends on
    // the cell alone, not on the order of the clips (which cells shared a
    // warp, or the previous rebuild's rotation); every lane of the warp
    // takes part, before any group returns
    const bool wr = live && status == 0;
    int mn = wr && g.gl < ne ? L.lab : 0x7fffffff;
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(kFull, mn, o));
    const unsigned at = g.ballot(wr && g.gl < ne && L.lab == mn);
    int src = g.gl + (at ? __ffs(at) - 1 : 0);
    if (src >= ne) src -= ne;
    const int lab = g.shfl(L.lab, src & (G - 1));
    if (!live) return;
    if (status == 2) {
        // out of lanes: queue the cell for the next wider pass (8 -> 16 -> 32
        // lanes), or from the 32-lane pass for the serial pass
        if (g.gl == 0) {
            if (G == 8) {
                int q = atomicAdd(a.ovf_n + 3, 1);
                a.ovf0_list[q] = s;
            } else if (G == 16) {
                int q = atomicAdd(a.ovf_n, 1);
                a.ovf_list[q] = s;
            } else {
                int q = atomicAdd(a.ovf_n + 1, 1);
                a.ovf2_list[q] = s;
            }
            if (P.debug) atomicAdd(&V.ctrl->cnt.vor_wide, 1ull);
        }
        return;
    }
    if (status != 0) {
        if (g.gl == 0) {
            a.ring_n[s] = 0;
            a.cellR[s] = 0.0f;
        }
        return;
    }
    if (g.gl < ne) a.ring[(size_t)s * kRingCap + g.gl] = lab;
    if (g.gl == 0) {
        a.ring_n[s] = (uint8_t)ne;
        a.cellR[s] = Rmax;
    }
}

// main pass: G lanes per cell, 32 / G cells per warp.  In a batch the cells
// of a warp lie in one chunk, hence in one mesh.
template <typename T, int G, bool B>
__global__ void __launch_bounds__(kVoroThreads, TRIME_VORO_MINB) k_voronoi(const __grid_constant__ IterArgs<T> a) {
    if (!B && skip_rebuild(a.V.ctrl, a.force)) return;
    __shared__ float4 stage_all[kVoroThreads / G][kStageCap];
    Grp<G> g;
    int lane = threadIdx.x & 31;
    g.gl = lane & (G - 1);
    g.goff = lane & ~(G - 1);
    constexpr int cpw = 32 / G;  // cells per warp
    int wib = threadIdx.x >> 5;
    int nwarps = gridDim.x * (kVoroThreads / 32);
    float4* stage = stage_all[threadIdx.x / G];
    for (int w = blockIdx.x * (kVoroThreads / 32) + wib; w * cpw < a.n; w += nwarps) {
        const MeshView& V = mesh_of<B>(a, w * cpw);
        if (B && skip_rebuild(V.ctrl, a.force)) continue;
        int s = w * cpw + lane / G;
        bool ok = s < a.n && (!B || s - V.soff < V.n);
        voronoi_cell<T, G, !B>(a, V, ok ? s : -1, g, stage);
    }
}

// wider pass over the cells a narrower one could not hold: G lanes per cell,
// the cells taken from a queue (the 8-lane pass's for G = 16, the 16-lane
// pass's for G = 32)
template <typename T, int G, bool B>
__global__ void __launch_bounds__(kVoroThreads, TRIME_VORO_MINB) k_voronoi_wide(const __grid_constant__ IterArgs<T> a) {
    if (!B && skip_rebuild(a.V.ctrl, a.force)) return;
    __shared__ float4 stage_all[kVoroThreads / G][kStageCap];
    Grp<G> g;
    int lane = threadIdx.x & 31;
    g.gl = lane & (G - 1);
    g.goff = lane & ~(G - 1);
    constexpr int cpw = 32 / G;
    const int32_t* list = G == 16 ? a.ovf0_list : a.ovf_list;
    int n = G == 16 ? a.ovf_n[3] : a.ovf_n[0];
    int wib = threadIdx.x >> 5;
    int nw = gridDim.x * (kVoroThreads / 32);
    float4* stage = stage_all[threadIdx.x / G];
    for (int w = blockIdx.x * (kVoroThreads / 32) + wib; w * cpw < n; w += nw) {
        int i = w * cpw + lane / G;
        int s = i < n ? list[i] : -1;
        // the cells of one warp may belong to different meshes of a batch:
        // each group reads its own mesh's view
        voronoi_cell<T, G, !B>(a, mesh_of<B>(a, s < 0 ? list[w * cpw] : s), s, g, stage);
    }
}

// ------------------------------------------------------------------ serial pass
// A cell with more than 32 edges (a sparse region bordering a dense one, e.g.
// a coarse boundary cell facing other parts of the shape across a narrow gap)
// is built by one thread with the same vertices, cut decisions, single-run
// rule and candidate order (bucket ring by bucket ring, nearest first within
// a staged set) as the warp passes; its polygon (up to kRingCap edges) and
// staged candidates live in shared memory.
constexpr int kSerialThreads = 16;
constexpr int kSerialStage = 96;

// edge as (nx, ny, s, label bits)
__device__ __forceinline__ Lane edge_vertex(const float4& e, const float4& f, float RB) {
    Lane L;
    L.nx = e.x;
    L.ny = e.y;
    L.s = e.z;
    L.lab = __float_as_int(e.w);
    L.bb = false;
    L.M = L.Qx = L.Qy = L.PM = L.PQx = L.PQy = 0.0f;
    make_vertex(L, f.x, f.y, f.z, __float_as_int(f.w), RB);
    return L;
}

// clip_by for one thread: 0 ok / no-op, 1 empty cell, 2 more than CAP edges
template <typename T, int CAP>
__device__ int clip_serial(float4* E, int& ne, float nx, float ny, float s, int lab, bool bisector, float RB,
                           const IterArgs<T>& a, const CellCtx& ctx) {
    // cut flags: one bit per vertex, in CAP / 64 words
    unsigned long long mw[(CAP + 63) / 64];
    for (int w = 0; w < (CAP + 63) / 64; w++) mw[w] = 0;
    auto cutv = [&](int t) { return (mw[t >> 6] >> (t & 63)) & 1ull; };
    for (int t = 0; t < ne; t++) {
        Lane L = edge_vertex(E[t], E[t + 1 == ne ? 0 : t + 1], RB);
        bool cut;
        if (bisector && L.bb) {
            float cl = 2.0f * s;
            float lam = fmaf(nx, L.Qx, fmaf(ny, L.Qy, cl * L.M));
            float P = fabsf(nx) * L.PQx + fabsf(ny) * L.PQy + cl * L.PM;
            float bound = 32.0f * kEps * P;
            if (P > 1e-30f && lam < -bound) cut = true;
            else if (P > 1e-30f && lam > bound) cut = false;
            else cut = exact_cut<T>(a, ctx, L.lab, L.nlab, lab);
        } else {
            cut = nx * L.vx + ny * L.vy > s;
        }
        if (cut) mw[t >> 6] |= 1ull << (t & 63);
    }
    int ncut = 0;
    for (int t = 0; t < ne; t++) ncut += (int)cutv(t);
    if (ncut == 0) return 0;
    if (ncut == ne) return 1;
    int starts = 0, sidx = -1;
    for (int t = 0; t < ne; t++) {
        int p = t == 0 ? ne - 1 : t - 1;
        if (cutv(t) && !cutv(p)) {
            starts++;
            if (sidx < 0) sidx = t;
        }
    }
    if (starts != 1) atomicAdd(&ctx.ctrl->cnt.clip_inconsistent, 1ull);
    int eidx = sidx;
    while (cutv(eidx)) eidx = eidx + 1 == ne ? 0 : eidx + 1;
    int k = sidx - eidx + 1;  // kept edges E_e .. E_s
    if (k <= 0) k += ne;
    if (k + 1 > CAP) return 2;
    // rotate E_e to position 0 in place (three reversals), then append
    auto rev = [&](int i, int j) {
        for (; i < j; i++, j--) {
            float4 x = E[i];
            E[i] = E[j];
            E[j] = x;
        }
    };
    if (eidx > 0) {
        rev(0, eidx - 1);
        rev(eidx, ne - 1);
        rev(0, ne - 1);
    }
    E[k] = make_float4(nx, ny, s, __int_as_float(lab));
    ne = k + 1;
    return 0;
}

template <typename T>
__device__ float serial_rmax(const float4* E, int ne, float RB) {
    float r = 0.0f;
    for (int t = 0; t < ne; t++) r = fmaxf(r, edge_vertex(E[t], E[t + 1 == ne ? 0 : t + 1], RB).vR);
    return r;
}

// builds cell s with at most CAP edges; the ring goes to out_ring / *out_len
// (and cellR); returns the status (2: more than CAP edges)
template <typename T, int CAP>
__device__ int voronoi_cell_serial(const IterArgs<T>& a, const MeshView& V, int s, float4* E, float4* C,
                                   int32_t* out_ring, int32_t* out_len) {
    const DevParams& P = V.P;
    const float INF = __int_as_float(0x7f800000);
    const float4 pi4 = a.pf[s];
    CellCtx ctx;
    ctx.ctrl = V.ctrl;
    ctx.si = s;
    ctx.dbg = P.debug;
    const float xf = (pi4.x - P.bx0f) + pi4.y, yf = (pi4.z - P.by0f) + pi4.w;
    const float Wf = P.Wf, Hf = P.Hf;
    float RB, mb;
    int ne;
    if (P.bounded) {
        float S = a.pS[s];
        float SB = S * (17.0f / 16.0f);
        RB = SB * 1.0824459f * 1.0001f;
        mb = S * (1.0f / 16.0f);
        const float c8[8] = {1.f, 0.70710678f, 0.f, -0.70710678f, -1.f, -0.70710678f, 0.f, 0.70710678f};
        for (int t = 0; t < 8; t++) E[t] = make_float4(c8[t], c8[(t + 6) & 7], SB, __int_as_float(oct_label(t)));
        ne = 8;
    } else {
        mb = 0.125f * (Wf > Hf ? Wf : Hf);
        RB = (sqrtf(Wf * Wf + Hf * Hf) + 4.0f * mb) * 1.0001f;
        ne = 4;
        for (int b = 0; b < 4; b++) {
            int bs = b == 0 ? 2 : (b == 1 ? 1 : (b == 2 ? 3 : 0));
            float nx = bs == 0 ? -1.f : (bs == 1 ? 1.f : 0.f);
            float ny = bs == 2 ? -1.f : (bs == 3 ? 1.f : 0.f);
            float sb = bs == 0 ? xf + mb : bs == 1 ? (Wf - xf) + mb : bs == 2 ? yf + mb : (Hf - yf) + mb;
            E[b] = make_float4(nx, ny, sb, __int_as_float(box_label(bs)));
        }
    }
    int status = 0;
    if (P.bounded) {
        for (int b = 0; b < 4 && status == 0; b++) {
            float nx = b == 0 ? -1.f : (b == 1 ? 1.f : 0.f);
            float ny = b == 2 ? -1.f : (b == 3 ? 1.f : 0.f);
            float sb = b == 0 ? xf + mb : b == 1 ? (Wf - xf) + mb : b == 2 ? yf + mb : (Hf - yf) + mb;
            status = clip_serial<T, CAP>(E, ne, nx, ny, sb, box_label(b), false, RB, a, ctx);
        }
    }
    float Rmax = status == 0 ? serial_rmax<T>(E, ne, RB) : 0.0f;
    int bxi, byi;
    bucket_of(P, pi4.x, pi4.z, bxi, byi);
    const float bsx = P.bsxf, bsy = P.bsyf;
    const float bmargin = P.bmargf + 4e-6f * (1.0f + fabsf(xf) + fabsf(yf));
    bool done = status != 0;
    int nst = 0;
    // apply the staged candidates nearest first
    auto flush = [&]() {
        unsigned long long used0 = 0, used1 = 0;
        while (!done) {
            float best = INF;
            int bi = -1;
            for (int q = 0; q < nst; q++) {
                bool u = q < 64 ? (used0 >> q) & 1ull : (used1 >> (q - 64)) & 1ull;
                if (!u && C[q].z < best) {
                    best = C[q].z;
                    bi = q;
                }
            }
            if (bi < 0 || !(best < 4.0f * Rmax * Rmax * 1.0001f)) break;
            if (bi < 64) used0 |= 1ull << bi;
            else used1 |= 1ull << (bi - 64);
            float4 c = C[bi];
            int ne0 = ne;
            int st = clip_serial<T, CAP>(E, ne, c.x, c.y, 0.5f * c.z, __float_as_int(c.w), true, RB, a, ctx);
            if (P.debug) {
                atomicAdd(&V.ctrl->cnt.vor_picks, 1ull);
                if (ne != ne0 || st) atomicAdd(&V.ctrl->cnt.vor_cuts, 1ull);
            }
            if (st) {
                status = st;
                done = true;
            } else if (ne != ne0) {
                Rmax = serial_rmax<T>(E, ne, RB);
            }
        }
        nst = 0;
    };
    for (int r = 1; !done; r++) {
        int nr = r == 1 ? 5 : 4 * r;
        for (int k = 0; k < nr && !done; k++) {
            int row, c0, c1;
            if (r == 1) {
                row = k < 3 ? byi : (k == 3 ? byi - 1 : byi + 1);
                c0 = k == 0 ? bxi : (k == 1 ? bxi - 1 : (k == 2 ? bxi + 1 : bxi - 1));
                c1 = k == 0 ? bxi : (k == 1 ? bxi - 1 : (k == 2 ? bxi + 1 : bxi + 1));
                if (k == 1 && c0 < 0) c0 = 1, c1 = 0;
                if (k == 2 && c1 >= P.nbx) c0 = 1, c1 = 0;
            } else if (k < 2) {
                row = k == 0 ? byi - r : byi + r;
                c0 = bxi - r;
                c1 = bxi + r;
            } else {
                int kk = k - 2;
                row = byi - r + 1 + (kk >> 1);
                c0 = c1 = (kk & 1) ? bxi + r : bxi - r;
            }
            c0 = c0 < 0 ? 0 : c0;
            c1 = c1 >= P.nbx ? P.nbx - 1 : c1;
            if (row < 0 || row >= P.nby || c0 > c1) continue;
            int lo = a.bstart[V.boff + row * P.nbx + c0], hi = a.bstart[V.boff + row * P.nbx + c1 + 1];
            for (int cs = lo; cs < hi && !done; cs++) {
                if (cs == s || a.dom[cs]) continue;
                float4 pj4 = a.pf[cs];
                float dx = ff_diff(pj4.x, pj4.y, pi4.x, pi4.y);
                float dy = ff_diff(pj4.z, pj4.w, pi4.z, pi4.w);
                float d2 = dx * dx + dy * dy;
                if (sizeof(T) == 8 && d2 < 9.094947e-13f) {
                    const float2 e = close_diff<T>(a.srt.x, a.srt.y, cs, a.srt.x[s], a.srt.y[s]);
                    dx = e.x;
                    dy = e.y;
                    d2 = dx * dx + dy * dy;
                }
                if (!(d2 < 4.0f * Rmax * Rmax * 1.0001f)) continue;
                if (nst == kSerialStage) flush();
                C[nst++] = make_float4(dx, dy, d2, __int_as_float(cs));
            }
        }
        flush();
        if (!done) {
            float dmin = INF;
            if (bxi - r > 0) dmin = fminf(dmin, xf - (float)(bxi - r) * bsx);
            if (bxi + r < P.nbx - 1) dmin = fminf(dmin, (float)(bxi + r + 1) * bsx - xf);
            if (byi - r > 0) dmin = fminf(dmin, yf - (float)(byi - r) * bsy);
            if (byi + r < P.nby - 1) dmin = fminf(dmin, (float)(byi + r + 1) * bsy - yf);
            bool all = bxi - r <= 0 && bxi + r >= P.nbx - 1 && byi - r <= 0 && byi + r >= P.nby - 1;
            if (all || 2.0f * Rmax * 1.0001f < dmin - bmargin) done = true;
        }
    }
    if (status != 0) {
        *out_len = 0;
        a.cellR[s] = 0.0f;
        return status;
    }
    for (int t = 0; t < ne; t++) out_ring[t] = __float_as_int(E[t].w);
    *out_len = ne;
    a.cellR[s] = Rmax;
    return 0;
}

template <typename T, bool B>
__global__ void __launch_bounds__(kSerialThreads) k_voronoi_serial(const __grid_constant__ IterArgs<T> a) {
    if (!B && skip_rebuild(a.V.ctrl, a.force)) return;
    __shared__ float4 edges[kSerialThreads][kRingCap + 1];
    __shared__ float4 stage[kSerialThreads][kSerialStage];
    int n = a.ovf_n[1];
    for (int i = blockIdx.x * kSerialThreads + threadIdx.x; i < n; i += gridDim.x * kSerialThreads) {
        int s = a.ovf2_list[i];
        const MeshView& V = mesh_of<B>(a, s);
        int32_t len;
        int st = voronoi_cell_serial<T, kRingCap>(a, V, s, edges[threadIdx.x], stage[threadIdx.x],
                                                   a.ring + (size_t)s * kRingCap, &len);
        a.ring_n[s] = (uint8_t)len;
        if (st == 2) {
            // more edges than a ring row holds: a guard trip, and the cell is
            // listed for the big-cell pass of the medial points
            atomicAdd(&V.ctrl->cnt.ring_overflow, 1ull);
            if (a.ovf3_list) a.ovf3_list[atomicAdd(a.ovf_n + 2, 1)] = s;
        }
    }
}

// cells beyond kRingCap edges, rebuilt on request (single mesh): polygon and
// staged candidates in global scratch, rings of up to kBigCap edges
constexpr int kBigCap = kBigRing;
constexpr size_t kBigScratch = kBigScratchF4;  // float4 per cell
static_assert(kBigScratch == (size_t)kBigCap + 1 + kSerialStage, "scratch layout");

template <typename T>
__global__ void __launch_bounds__(32) k_voronoi_big(const __grid_constant__ IterArgs<T> a, int32_t n,
                                                    float4* scratch, int32_t* rings, int32_t* lens) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int s = a.ovf3_list[i];
        float4* E = scratch + (size_t)i * kBigScratch;
        voronoi_cell_serial<T, kBigCap>(a, a.V, s, E, E + kBigCap + 1, rings + (size_t)i * kBigCap, lens + i);
    }
}

template <typename T>
void launch_voronoi_big(const IterArgs<T>& a, int32_t n, float4* scratch, int32_t* rings, int32_t* lens,
                        cudaStream_t st) {
    if (n > 0) k_voronoi_big<T><<<(n + 31) / 32, 32, 0, st>>>(a, n, scratch, rings, lens);
}

// lanes = 8: four cells per warp, then the 16- and 32-lane passes for the
// queued cells; lanes = 16: two cells per warp plus the 32-lane pass;
// lanes = 32: one cell per warp.  The serial pass follows in every case.
template <typename T, bool B>
void launch_voronoi_impl(const IterArgs<T>& a, int lanes, cudaStream_t st) {
    cudaMemsetAsync(a.ovf_n, 0, 4 * sizeof(int32_t), st);
    int cpb = kVoroThreads / lanes;  // cells per block
    int g = (a.n + cpb - 1) / cpb;
    if (g < 1) g = 1;
    if (lanes == 32) {
        k_voronoi<T, 32, B><<<g, kVoroThreads, 0, st>>>(a);
    } else if (lanes == 16) {
        k_voronoi<T, 16, B><<<g, kVoroThreads, 0, st>>>(a);
        k_voronoi_wide<T, 32, B><<<152 * 2, kVoroThreads, 0, st>>>(a);
    } else {
        k_voronoi<T, 8, B><<<g, kVoroThreads, 0, st>>>(a);
        k_voronoi_wide<T, 16, B><<<152 * TRIME_VORO_MINB, kVoroThreads, 0, st>>>(a);
        k_voronoi_wide<T, 32, B><<<152 * 2, kVoroThreads, 0, st>>>(a);
    }
    k_voronoi_serial<T, B><<<152, kSerialThreads, 0, st>>>(a);
}

}  // namespace trime
