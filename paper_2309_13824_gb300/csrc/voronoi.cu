// voronoi.cu -- a2: bounded Voronoi cell of every point by half-plane
// clipping (TriMe++ Sec. 2.1 Fig. 3, cell-based approach; Sec. 4.1 octagon
// bound of span S = fac_voro_bound * h_i).
//
// One warp per cell.  The convex polygon lives in the warp, one edge per lane
// (<= 32 edges): lane t holds edge E_t as a half-plane n.u <= s (u relative to
// the generator) and the vertex V_t = E_t cap E_{t+1}.  Candidates come from
// the bucket grid ring by ring, are loaded one per lane, filtered by the
// security radius (a point farther than twice the largest vertex distance
// cannot cut) and applied nearest first.  A clip classifies every vertex in
// parallel, finds the single run of cut vertices with two ballots and
// rotates the edge list with shuffles.
//
// Exactness: a vertex where two bisectors meet is the circumcentre of
// (i, j, k); the candidate l cuts it iff det4(i,j,k,l) > 0 (l inside that
// circle), decided by a float filter with a proven error bound, then an FP64
// filter, then exact expansion arithmetic with symbolic perturbation.  Other
// vertices involve a bounding line; they are tested in float.  The bounding
// octagon and box used here are enlarged by 1/16 of S over the region Reg_i
// that the emission test reads, so those float decisions cannot change which
// Delaunay triangles have their circumcentre inside Reg_i.
#include "exact.cuh"
#include "kernels.cuh"

namespace trime {

constexpr float kEps = 5.9604645e-8f;  // 2^-24
constexpr unsigned kFull = 0xffffffffu;
constexpr int kStageCap = 160;  // staged candidates per warp (16 bytes each)

struct Lane {
    float nx, ny, s;      // edge half-plane n.u <= s
    int lab;              // >= 0 bisector (neighbour slot) / < 0 bounding line
    float vx, vy, vR;     // vertex with the next edge and an upper bound of |V|
    int nlab;             // next edge's label
    bool bb;              // vertex of two bisectors
    float Qx, Qy, M;      // det4 filter terms of a bisector-bisector vertex
    float PQx, PQy, PM;   // and their absolute-value permanents
};

__device__ __forceinline__ void make_vertex(Lane& L, float nx2, float ny2, float s2, int lab2, float RB) {
    float D = L.nx * ny2 - L.ny * nx2;
    float px = L.s * ny2 - s2 * L.ny, py = s2 * L.nx - L.s * nx2;
    float ux = px / D, uy = py / D;
    float r = sqrtf(ux * ux + uy * uy);
    float perm = fabsf(L.s * ny2) + fabsf(s2 * L.ny) + fabsf(s2 * L.nx) + fabsf(L.s * nx2) +
                 r * (fabsf(L.nx * ny2) + fabsf(L.ny * nx2));
    float err = 64.0f * kEps * perm / fabsf(D);
    bool ok = (D != 0.0f) && (r + err < RB);  // false for NaN as well
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
}

// vertex of this lane with the next lane's edge (all lanes participate)
__device__ __forceinline__ void lane_vertex(Lane& L, int ne, int lane, float RB, bool active) {
    int nxt = lane + 1 >= ne ? 0 : lane + 1;
    float nx2 = __shfl_sync(kFull, L.nx, nxt), ny2 = __shfl_sync(kFull, L.ny, nxt);
    float s2 = __shfl_sync(kFull, L.s, nxt);
    int lab2 = __shfl_sync(kFull, L.lab, nxt);
    if (active && lane < ne) make_vertex(L, nx2, ny2, s2, lab2, RB);
}

template <typename T>
struct CellCtx {
    const T* x;
    const T* y;
    const int32_t* id;
    DevCtrl* ctrl;
    double pix, piy;
    int idi;
};

// exact decision for vertex (j, k) of cell i against candidate l: FP64 filter,
// then expansion arithmetic with symbolic perturbation
template <typename T>
__device__ __noinline__ bool exact_cut(const CellCtx<T>& c, int sj, int sk, int sl) {
    double pi[2] = {c.pix, c.piy};
    double pj[2] = {(double)c.x[sj], (double)c.y[sj]};
    double pk[2] = {(double)c.x[sk], (double)c.y[sk]};
    double pl[2] = {(double)c.x[sl], (double)c.y[sl]};
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
    int d = incircle_sos(pi, c.idi, pj, c.id[sj], pk, c.id[sk], pl, c.id[sl]);
    if (o == kExactFail || d == kExactFail) {
        atomicAdd(&c.ctrl->cnt.exact_overflow, 1ull);
        return false;
    }
    return d * o > 0;
}

// Clip the warp's polygon by n.u <= s (label lab).  bisector: a neighbour's
// bisector (n = d, s = |d|^2/2).  Returns 0 ok, 1 empty, 2 overflow.
template <typename T>
__device__ int clip_by(Lane& L, int& ne, float nx, float ny, float s, int lab, bool bisector, float RB, int lane,
                       const CellCtx<T>& ctx) {
    bool cut = false;
    if (lane < ne) {
        if (bisector && L.bb) {
            float cl = 2.0f * s;
            float lam = fmaf(nx, L.Qx, fmaf(ny, L.Qy, cl * L.M));
            float P = fabsf(nx) * L.PQx + fabsf(ny) * L.PQy + cl * L.PM;
            float bound = 32.0f * kEps * P;
            if (P > 1e-30f && lam < -bound) cut = true;
            else if (P > 1e-30f && lam > bound) cut = false;
            else cut = exact_cut<T>(ctx, L.lab, L.nlab, lab);
        } else {
            cut = nx * L.vx + ny * L.vy > s;
        }
    }
    unsigned m = __ballot_sync(kFull, cut);
    if (m == 0) return 0;
    unsigned full = ne >= 32 ? kFull : ((1u << ne) - 1u);
    if ((m & full) == full) return 1;
    int prevl = lane == 0 ? ne - 1 : lane - 1;
    bool pcut = (m >> (prevl & 31)) & 1u;
    unsigned starts = __ballot_sync(kFull, lane < ne && cut && !pcut);
    unsigned ends = __ballot_sync(kFull, lane < ne && !cut && pcut);
    if (__popc(starts) != 1 && lane == 0) atomicAdd(&ctx.ctrl->cnt.clip_inconsistent, 1ull);
    int sidx = __ffs(starts) - 1;
    unsigned after = sidx >= 31 ? 0u : (ends >> (sidx + 1)) << (sidx + 1);
    int eidx = after ? __ffs(after) - 1 : __ffs(ends) - 1;
    int k = (sidx - eidx + ne) % ne + 1;  // kept edges E_e .. E_s
    int nn = k + 1;
    if (nn > kRingCap) return 2;
    int src = (eidx + lane) % ne;
    Lane R;
    R.nx = __shfl_sync(kFull, L.nx, src);
    R.ny = __shfl_sync(kFull, L.ny, src);
    R.s = __shfl_sync(kFull, L.s, src);
    R.lab = __shfl_sync(kFull, L.lab, src);
    R.vx = __shfl_sync(kFull, L.vx, src);
    R.vy = __shfl_sync(kFull, L.vy, src);
    R.vR = __shfl_sync(kFull, L.vR, src);
    R.nlab = __shfl_sync(kFull, L.nlab, src);
    R.bb = __shfl_sync(kFull, (int)L.bb, src) != 0;
    R.Qx = __shfl_sync(kFull, L.Qx, src);
    R.Qy = __shfl_sync(kFull, L.Qy, src);
    R.M = __shfl_sync(kFull, L.M, src);
    R.PQx = __shfl_sync(kFull, L.PQx, src);
    R.PQy = __shfl_sync(kFull, L.PQy, src);
    R.PM = __shfl_sync(kFull, L.PM, src);
    if (lane < k) L = R;
    if (lane == k) {
        L.nx = nx;
        L.ny = ny;
        L.s = s;
        L.lab = lab;
    }
    ne = nn;
    lane_vertex(L, ne, lane, RB, lane == k - 1 || lane == k);
    return 0;
}

template <typename T>
__device__ __forceinline__ void finish_cell(const IterArgs<T>& a, int s, int lane, const Lane& L, int ne, float R) {
    if (lane < ne) a.ring[(size_t)s * kRingCap + lane] = L.lab;
    if (lane == 0) {
        a.ring_n[s] = (uint8_t)ne;
        a.cellR[s] = R;
    }
}

template <typename T>
__device__ void voronoi_cell(const IterArgs<T>& a, int s, int lane) {
    const DevParams& P = a.P;
    if (a.dom[s]) {
        if (lane == 0) {
            a.ring_n[s] = 0;
            a.cellR[s] = 0.0f;
        }
        return;
    }
    T xi = a.srt.x[s], yi = a.srt.y[s];
    CellCtx<T> ctx;
    ctx.x = a.srt.x;
    ctx.y = a.srt.y;
    ctx.id = a.srt.id;
    ctx.ctrl = a.ctrl;
    ctx.pix = (double)xi;
    ctx.piy = (double)yi;
    ctx.idi = a.srt.id[s];
    double W = P.bx1 - P.bx0, H = P.by1 - P.by0;
    float RB, mb;
    Lane L;
    L.bb = false;
    L.vR = 0.0f;
    int ne;
    if (P.bounded) {
        float S = (float)(P.fac_voro_bound * a.gh[a.cell[s]]);
        float SB = S * (17.0f / 16.0f);
        RB = SB * 1.0824459f * 1.0001f;  // octagon circumradius SB / cos(pi/8)
        mb = S * (1.0f / 16.0f);
        const float c8[8] = {1.f, 0.70710678f, 0.f, -0.70710678f, -1.f, -0.70710678f, 0.f, 0.70710678f};
        int t = lane & 7;
        L.nx = c8[t];
        L.ny = c8[(t + 6) & 7];
        L.s = SB;
        L.lab = oct_label(t);
        ne = 8;
    } else {
        mb = (float)(0.125 * (W > H ? W : H));
        RB = (float)((sqrt(W * W + H * H) + 4.0 * mb) * 1.0001);
        ne = 4;  // enlarged box, CCW: bottom, right, top, left
        int b = lane & 3;
        const int bside[4] = {2, 1, 3, 0};
        int bs = bside[b];
        L.nx = bs == 0 ? -1.f : (bs == 1 ? 1.f : 0.f);
        L.ny = bs == 2 ? -1.f : (bs == 3 ? 1.f : 0.f);
        L.s = bs == 0 ? (float)(ctx.pix - (P.bx0 - mb)) : bs == 1 ? (float)((P.bx1 + mb) - ctx.pix)
            : bs == 2 ? (float)(ctx.piy - (P.by0 - mb)) : (float)((P.by1 + mb) - ctx.piy);
        L.lab = box_label(bs);
    }
    lane_vertex(L, ne, lane, RB, true);
    if (P.bounded) {
        for (int b = 0; b < 4; b++) {
            float nx = b == 0 ? -1.f : (b == 1 ? 1.f : 0.f);
            float ny = b == 2 ? -1.f : (b == 3 ? 1.f : 0.f);
            float sb = b == 0 ? (float)(ctx.pix - (P.bx0 - mb)) : b == 1 ? (float)((P.bx1 + mb) - ctx.pix)
                     : b == 2 ? (float)(ctx.piy - (P.by0 - mb)) : (float)((P.by1 + mb) - ctx.piy);
            clip_by<T>(L, ne, nx, ny, sb, box_label(b), false, RB, lane, ctx);
        }
    }
    float Rmax = warp_max(lane < ne ? L.vR : 0.0f);
    int bxi, byi;
    bucket_of(P, xi, yi, bxi, byi);
    const float xf = (float)(ctx.pix - P.bx0), yf = (float)(ctx.piy - P.by0);
    const float bsx = (float)P.bsx, bsy = (float)P.bsy;
    const float bmargin = (float)(1e-3 * (P.bsx > P.bsy ? P.bsx : P.bsy)) + 4e-6f * (1.0f + fabsf(xf) + fabsf(yf));
    const float INF = __int_as_float(0x7f800000);
    // per-warp staging buffer: candidates of the current ring, applied
    // nearest first across the whole staged set
    __shared__ float4 stage_all[kVoroThreads / 32][kStageCap];
    float4* stage = stage_all[threadIdx.x >> 5];
    int nst = 0;
    auto flush = [&]() -> int {
        while (true) {
            float best = INF;
            int bi = -1;
            float lim = 4.0f * Rmax * Rmax * 1.0001f;
            for (int q = lane; q < nst; q += 32) {
                float d2 = stage[q].z;
                if (d2 < lim && d2 < best) {
                    best = d2;
                    bi = q;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                float ob = __shfl_xor_sync(kFull, best, o);
                int oi = __shfl_xor_sync(kFull, bi, o);
                if (ob < best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (bi < 0) break;
            float4 c = stage[bi];
            __syncwarp();
            if (lane == 0) stage[bi].z = INF;
            __syncwarp();
            int st = clip_by<T>(L, ne, c.x, c.y, 0.5f * c.z, __float_as_int(c.w), true, RB, lane, ctx);
            if (st) return st;
            Rmax = warp_max(lane < ne ? L.vR : 0.0f);
        }
        nst = 0;
        __syncwarp();
        return 0;
    };
    for (int r = 1;; r++) {
        int nr = r == 1 ? 5 : 4 * r;
        for (int kb = 0; kb < nr; kb += 32) {
            int k = kb + lane;
            int lo = 0, hi = 0;
            if (k < nr) {
                int row, c0, c1;
                if (r == 1) {
                    // own bucket first, then its row neighbours, then the rows below / above
                    row = k < 3 ? byi : (k == 3 ? byi - 1 : byi + 1);
                    c0 = k == 0 ? bxi : (k == 1 ? bxi - 1 : (k == 2 ? bxi + 1 : bxi - 1));
                    c1 = k == 0 ? bxi : (k == 1 ? bxi - 1 : (k == 2 ? bxi + 1 : bxi + 1));
                    if (k == 1 && c0 < 0) c0 = 1, c1 = 0;            // no bucket left of the grid
                    if (k == 2 && c1 >= P.nbx) c0 = 1, c1 = 0;       // no bucket right of the grid
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
                if (row >= 0 && row < P.nby && c0 <= c1) {
                    lo = a.bstart[row * P.nbx + c0];
                    hi = a.bstart[row * P.nbx + c1 + 1];
                }
            }
            int cnt = hi - lo;
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            int total = __shfl_sync(kFull, incl, 31);
            int excl = incl - cnt;
            for (int q0 = 0; q0 < total; q0 += 32) {
                int q = q0 + lane;
                int ow = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    int pr = ow + step;
                    int ex = __shfl_sync(kFull, excl, pr);
                    if (ex <= q) ow = pr;
                }
                int olo = __shfl_sync(kFull, lo, ow);
                int oex = __shfl_sync(kFull, excl, ow);
                int slot = olo + (q - oex);
                bool valid = q < total && slot != s;
                float dx = 0.f, dy = 0.f, d2 = INF;
                if (valid) valid = !a.dom[slot];
                if (valid) {
                    T xj = a.srt.x[slot], yj = a.srt.y[slot];
                    dx = (float)(xj - xi);
                    dy = (float)(yj - yi);
                    d2 = dx * dx + dy * dy;
                }
                bool keep = valid && d2 < 4.0f * Rmax * Rmax * 1.0001f;
                unsigned km = __ballot_sync(kFull, keep);
                if (nst + __popc(km) > kStageCap) {
                    int st = flush();
                    if (st) {
                        if (st == 2 && lane == 0) atomicAdd(&a.ctrl->cnt.ring_overflow, 1ull);
                        if (lane == 0) {
                            a.ring_n[s] = 0;
                            a.cellR[s] = 0.0f;
                        }
                        return;
                    }
                    keep = keep && d2 < 4.0f * Rmax * Rmax * 1.0001f;
                    km = __ballot_sync(kFull, keep);
                }
                if (keep) stage[nst + __popc(km & ((1u << lane) - 1u))] = make_float4(dx, dy, d2, __int_as_float(slot));
                nst += __popc(km);
                __syncwarp();
            }
        }
        int st = flush();
        if (st) {
            if (st == 2 && lane == 0) atomicAdd(&a.ctrl->cnt.ring_overflow, 1ull);
            if (lane == 0) {
                a.ring_n[s] = 0;
                a.cellR[s] = 0.0f;
            }
            return;
        }
        // nothing outside the (2r+1)^2 block can cut once it is beyond 2 Rmax
        float dmin = INF;
        if (bxi - r > 0) dmin = fminf(dmin, xf - (float)(bxi - r) * bsx);
        if (bxi + r < P.nbx - 1) dmin = fminf(dmin, (float)(bxi + r + 1) * bsx - xf);
        if (byi - r > 0) dmin = fminf(dmin, yf - (float)(byi - r) * bsy);
        if (byi + r < P.nby - 1) dmin = fminf(dmin, (float)(byi + r + 1) * bsy - yf);
        bool all = bxi - r <= 0 && bxi + r >= P.nbx - 1 && byi - r <= 0 && byi + r >= P.nby - 1;
        if (all || 2.0f * Rmax * 1.0001f < dmin - bmargin) break;
    }
    finish_cell(a, s, lane, L, ne, Rmax);
}

template <typename T>
__global__ void __launch_bounds__(kVoroThreads) k_voronoi(IterArgs<T> a) {
    if (!a.force && a.ctrl->terminated) return;
    int lane = threadIdx.x & 31;
    int wpb = blockDim.x >> 5;
    for (int s = blockIdx.x * wpb + (threadIdx.x >> 5); s < a.n; s += gridDim.x * wpb) voronoi_cell<T>(a, s, lane);
}

template <typename T>
void launch_voronoi(const IterArgs<T>& a, cudaStream_t st) {
    int wpb = kVoroThreads / 32;
    int g = (a.n + wpb - 1) / wpb;
    if (g < 1) g = 1;
    k_voronoi<T><<<g, kVoroThreads, 0, st>>>(a);
}

template void launch_voronoi<double>(const IterArgs<double>&, cudaStream_t);
// device exact predicates on explicit queries (verification hook)
__global__ void k_predicates(const double* pts, const int32_t* ids, int32_t nq, int32_t* o_out, int32_t* c_out) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const double* p = pts + 8 * (size_t)q;
    const int32_t* id = ids + 4 * (size_t)q;
    o_out[q] = orient_exact(p, p + 2, p + 4);
    c_out[q] = incircle_sos(p, id[0], p + 2, id[1], p + 4, id[2], p + 6, id[3]);
}

void launch_predicates(const double* pts, const int32_t* ids, int32_t nq, int32_t* o_out, int32_t* c_out,
                       cudaStream_t st) {
    if (nq > 0) k_predicates<<<(nq + 127) / 128, 128, 0, st>>>(pts, ids, nq, o_out, c_out);
}
template void launch_voronoi<float>(const IterArgs<float>&, cudaStream_t);

}  // namespace trime
