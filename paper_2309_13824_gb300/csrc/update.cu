// update.cu -- a5/a6/a7 and the a8 finalisation (TriMe++ Sec. 2.2-2.4, 4.2-4.3).
//
// One thread per cell computes the raw new position -- DistMesh: forward
// Euler with the spring forces of its valid edges (Eqs. 2-5), gathered from
// its own ring so no atomics are needed; CVD: the density-weighted centroid
// of its bounded cell by adaptive longest-edge-bisection quadrature (Eq. 6,
// Sec. 4.2) -- then clamps the move, classifies the point on the geometry
// grid and projects it back by sphere tracing or damped Newton (Sec. 4.3).
// The statistics kernels finalise the quality 1/2-means (Eq. 12), fac_mu
// (Eq. 3), the hybrid switch (Sec. 4.2) and the termination tests (Sec. 4).
#include "ff.cuh"
#include "kernels.cuh"
#include "treat.cuh"

namespace trime {

constexpr int kPolyCap = kRingCap + 16;  // ring edges plus the octagon and box clips

// ------------------------------------------------------------------ CVD centroid
template <typename T>
struct Poly {
    T nx[kPolyCap], ny[kPolyCap], s[kPolyCap];
    int m;
};

template <typename T>
__device__ __forceinline__ void isect(const Poly<T>& P, int a, int b, T& ux, T& uy) {
    T D = P.nx[a] * P.ny[b] - P.ny[a] * P.nx[b];
    ux = (P.s[a] * P.ny[b] - P.s[b] * P.ny[a]) / D;
    uy = (P.s[b] * P.nx[a] - P.s[a] * P.nx[b]) / D;
}

// clip by n.u <= s keeping one run (Sutherland-Hodgman on labelled edges)
template <typename T>
__device__ void clip_poly(Poly<T>& P, T nx, T ny, T s) {
    int m = P.m;
    if (m == 0) return;
    unsigned long long cut = 0;
    for (int t = 0; t < m; t++) {
        T ux, uy;
        isect(P, t, t + 1 == m ? 0 : t + 1, ux, uy);
        if (nx * ux + ny * uy > s) cut |= 1ull << t;
    }
    if (!cut) return;
    unsigned long long full = m >= 64 ? ~0ull : ((1ull << m) - 1);
    if ((cut & full) == full) { P.m = 0; return; }
    int st = -1;
    for (int t = 0; t < m && st < 0; t++)
        if (((cut >> t) & 1) && !((cut >> (t == 0 ? m - 1 : t - 1)) & 1)) st = t;
    int e = st;
    while ((cut >> e) & 1) e = e + 1 == m ? 0 : e + 1;
    T tnx[kPolyCap], tny[kPolyCap], ts[kPolyCap];
    int k = 0;
    for (int t = e;; t = t + 1 == m ? 0 : t + 1) {
        tnx[k] = P.nx[t]; tny[k] = P.ny[t]; ts[k] = P.s[t];
        k++;
        if (t == st) break;
    }
    if (k + 1 > kPolyCap) { P.m = 0; return; }
    tnx[k] = nx; tny[k] = ny; ts[k] = s;
    k++;
    for (int t = 0; t < k; t++) { P.nx[t] = tnx[t]; P.ny[t] = tny[t]; P.s[t] = ts[t]; }
    P.m = k;
}

// one-point rule on the leaves of the longest-edge bisection tree of given
// depth under the triangle (0, v1, v2) (relative to the generator)
template <typename T>
__device__ void level_sum(const MeshView& V, T gx, T gy, T v1x, T v1y, T v2x, T v2y, int depth, T& W, T& WX,
                          T& WY) {
    T st[9][6];
    int sd[9];
    int sp = 0;
    st[0][0] = 0; st[0][1] = 0; st[0][2] = v1x; st[0][3] = v1y; st[0][4] = v2x; st[0][5] = v2y;
    sd[0] = depth;
    sp = 1;
    while (sp > 0) {
        sp--;
        T q0x = st[sp][0], q0y = st[sp][1], q1x = st[sp][2], q1y = st[sp][3], q2x = st[sp][4], q2y = st[sp][5];
        int d = sd[sp];
        if (d == 0) {
            T A = (T)0.5 * ((q1x - q0x) * (q2y - q0y) - (q1y - q0y) * (q2x - q0x));
            T cx = (q0x + q1x + q2x) * (T)(1.0 / 3.0), cy = (q0y + q1y + q2y) * (T)(1.0 / 3.0);
            T mu = bilin<T>(V.siz, gx + cx, gy + cy);
            T w = A / (mu * mu);
            W += w;
            WX += w * cx;
            WY += w * cy;
            continue;
        }
        T L01 = (q1x - q0x) * (q1x - q0x) + (q1y - q0y) * (q1y - q0y);
        T L12 = (q2x - q1x) * (q2x - q1x) + (q2y - q1y) * (q2y - q1y);
        T L20 = (q0x - q2x) * (q0x - q2x) + (q0y - q2y) * (q0y - q2y);
        T ax = q0x, ay = q0y, bx = q1x, by = q1y, cx = q2x, cy = q2y, Lm = L01;
        if (L12 > Lm) { ax = q1x; ay = q1y; bx = q2x; by = q2y; cx = q0x; cy = q0y; Lm = L12; }
        if (L20 > Lm) { ax = q2x; ay = q2y; bx = q0x; by = q0y; cx = q1x; cy = q1y; }
        T mx = (ax + bx) * (T)0.5, my = (ay + by) * (T)0.5;
        // children (a, m, c) and (m, b, c); push the second first
        st[sp][0] = mx; st[sp][1] = my; st[sp][2] = bx; st[sp][3] = by; st[sp][4] = cx; st[sp][5] = cy;
        sd[sp] = d - 1;
        sp++;
        st[sp][0] = ax; st[sp][1] = ay; st[sp][2] = mx; st[sp][3] = my; st[sp][4] = cx; st[sp][5] = cy;
        sd[sp] = d - 1;
        sp++;
    }
}

// The same tree in float-float (FP64 mode): vertices relative to the
// generator, the generator as a float pair; the longest edge, the leaf areas,
// centroids, sizing and weights all carry about 48 bits.
__device__ void level_sum_ff(const MeshView& V, ff gx, ff gy, ff v1x, ff v1y, ff v2x, ff v2y, int depth, ff& W,
                             ff& WX, ff& WY) {
    const ff third{__int_as_float(0x3EAAAAAB), __int_as_float(0xB22AAAAB)};  // 1/3 to 2^-50
    ff st[9][6];
    int sd[9];
    const ff z{0.f, 0.f};
    st[0][0] = z; st[0][1] = z; st[0][2] = v1x; st[0][3] = v1y; st[0][4] = v2x; st[0][5] = v2y;
    sd[0] = depth;
    int sp = 1;
    while (sp > 0) {
        sp--;
        ff q0x = st[sp][0], q0y = st[sp][1], q1x = st[sp][2], q1y = st[sp][3], q2x = st[sp][4], q2y = st[sp][5];
        int d = sd[sp];
        if (d == 0) {
            ff A = ff_scale2(ff_sub(ff_mul(ff_sub(q1x, q0x), ff_sub(q2y, q0y)),
                                    ff_mul(ff_sub(q1y, q0y), ff_sub(q2x, q0x))), 0.5f);
            ff cx = ff_mul(ff_add(ff_add(q0x, q1x), q2x), third);
            ff cy = ff_mul(ff_add(ff_add(q0y, q1y), q2y), third);
            ff mu = bilin_ff(V.siz, ff_add(gx, cx), ff_add(gy, cy));
            ff w = ff_div(A, ff_mul(mu, mu));
            W = ff_add(W, w);
            WX = ff_add(WX, ff_mul(w, cx));
            WY = ff_add(WY, ff_mul(w, cy));
            continue;
        }
        ff e0x = ff_sub(q1x, q0x), e0y = ff_sub(q1y, q0y);
        ff e1x = ff_sub(q2x, q1x), e1y = ff_sub(q2y, q1y);
        ff e2x = ff_sub(q0x, q2x), e2y = ff_sub(q0y, q2y);
        ff L01 = ff_add(ff_mul(e0x, e0x), ff_mul(e0y, e0y));
        ff L12 = ff_add(ff_mul(e1x, e1x), ff_mul(e1y, e1y));
        ff L20 = ff_add(ff_mul(e2x, e2x), ff_mul(e2y, e2y));
        ff ax = q0x, ay = q0y, bx = q1x, by = q1y, cx = q2x, cy = q2y, Lm = L01;
        if (ff_gt(L12, Lm)) { ax = q1x; ay = q1y; bx = q2x; by = q2y; cx = q0x; cy = q0y; Lm = L12; }
        if (ff_gt(L20, Lm)) { ax = q2x; ay = q2y; bx = q0x; by = q0y; cx = q1x; cy = q1y; }
        ff mx = ff_scale2(ff_add(ax, bx), 0.5f), my = ff_scale2(ff_add(ay, by), 0.5f);
        st[sp][0] = mx; st[sp][1] = my; st[sp][2] = bx; st[sp][3] = by; st[sp][4] = cx; st[sp][5] = cy;
        sd[sp] = d - 1;
        sp++;
        st[sp][0] = ax; st[sp][1] = ay; st[sp][2] = mx; st[sp][3] = my; st[sp][4] = cx; st[sp][5] = cy;
        sd[sp] = d - 1;
        sp++;
    }
}

template <typename T>
__device__ void cvd_centroid(const IterArgs<T>& a, const MeshView& V, int s, int ne, const int* lab, T xi, T yi, T h,
                             T dprev, T& cx, T& cy, int& level, bool& capped) {
    const DevParams& P = V.P;
    cx = xi;
    cy = yi;
    level = 0;
    capped = false;
    if (ne < 3) return;
    Poly<T> poly;
    T W_ = (T)(P.bx1 - P.bx0), H_ = (T)(P.by1 - P.by0);
    T S = (T)P.fac_voro_bound * h;
    T SB = S * (T)(17.0 / 16.0);
    T mb = P.bounded ? S * (T)(1.0 / 16.0) : (T)0.125 * (W_ > H_ ? W_ : H_);
    T bl = xi - ((T)P.bx0 - mb), br = ((T)P.bx1 + mb) - xi, bb = yi - ((T)P.by0 - mb), bt = ((T)P.by1 + mb) - yi;
    for (int t = 0; t < ne; t++) {
        int l = lab[t];
        if (l >= 0) {
            T dx = a.srt.x[l] - xi, dy = a.srt.y[l] - yi;
            poly.nx[t] = dx; poly.ny[t] = dy; poly.s[t] = (T)0.5 * (dx * dx + dy * dy);
        } else if (l >= -8) {
            int k = -1 - l;
            const T c8[8] = {(T)1, (T)kRT, (T)0, -(T)kRT, (T)-1, -(T)kRT, (T)0, (T)kRT};
            poly.nx[t] = c8[k]; poly.ny[t] = c8[(k + 6) & 7]; poly.s[t] = SB;
        } else {
            int b = -9 - l;
            poly.nx[t] = b == 0 ? (T)-1 : (b == 1 ? (T)1 : (T)0);
            poly.ny[t] = b == 2 ? (T)-1 : (b == 3 ? (T)1 : (T)0);
            poly.s[t] = b == 0 ? bl : (b == 1 ? br : (b == 2 ? bb : bt));
        }
    }
    poly.m = ne;
    T R = (T)a.cellR[s];
    T dl = xi - (T)P.bx0, dr = (T)P.bx1 - xi, db = yi - (T)P.by0, dt_ = (T)P.by1 - yi;
    T dbox = fmin(fmin(dl, dr), fmin(db, dt_));
    bool inside = R * (T)1.0001 < dbox && (!P.bounded || R * (T)1.0001 < S);
    if (!inside) {
        if (P.bounded) {
            const T c8[8] = {(T)1, (T)kRT, (T)0, -(T)kRT, (T)-1, -(T)kRT, (T)0, (T)kRT};
            for (int k = 0; k < 8; k++) clip_poly(poly, c8[k], c8[(k + 6) & 7], S);
        }
        clip_poly(poly, (T)-1, (T)0, dl);
        clip_poly(poly, (T)1, (T)0, dr);
        clip_poly(poly, (T)0, (T)-1, db);
        clip_poly(poly, (T)0, (T)1, dt_);
    }
    int m = poly.m;
    if (m < 3) return;
    T vx[kPolyCap], vy[kPolyCap];
    T A = 0;
    for (int t = 0; t < m; t++) isect(poly, t, t + 1 == m ? 0 : t + 1, vx[t], vy[t]);
    for (int t = 0; t < m; t++) {
        int u = t + 1 == m ? 0 : t + 1;
        A += (T)0.5 * (vx[t] * vy[u] - vy[t] * vx[u]);
    }
    if (!(A > 0)) return;
    T E = sqrt(A) * fmax(dprev / h, (T)P.fac_end);
    int Lmax = P.quad_max_level;
    if (sizeof(T) == 8) {
        // FP64 mode: the quadrature in float-float (the vertices above stay FP64)
        const float4 pi4 = a.pf[s];
        const ff gx{pi4.x, pi4.y}, gy{pi4.z, pi4.w};
        ff fvx[kPolyCap], fvy[kPolyCap];
        for (int t = 0; t < m; t++) {
            fvx[t] = ff_from_d((double)vx[t]);
            fvy[t] = ff_from_d((double)vy[t]);
        }
        ff E2 = ff_from_d((double)(E * E));
        ff fpx{0.f, 0.f}, fpy{0.f, 0.f};
        for (int k = 1; k <= Lmax; k++) {
            ff W{0.f, 0.f}, WX{0.f, 0.f}, WY{0.f, 0.f};
            for (int t = 0; t < m; t++) {
                int u = t + 1 == m ? 0 : t + 1;
                level_sum_ff(V, gx, gy, fvx[t], fvy[t], fvx[u], fvy[u], k - 1, W, WX, WY);
            }
            if (!(W.h > 0.f)) return;
            ff ccx = ff_div(WX, W), ccy = ff_div(WY, W);
            ff dx = ff_sub(ccx, fpx), dy = ff_sub(ccy, fpy);
            bool conv = ff_gt(E2, ff_add(ff_mul(dx, dx), ff_mul(dy, dy)));
            if (conv || k == Lmax) {
                cx = xi + (T)ff_to_d(ccx);
                cy = yi + (T)ff_to_d(ccy);
                level = k;
                capped = !conv;
                return;
            }
            fpx = ccx;
            fpy = ccy;
        }
        return;
    }
    T px = 0, py = 0;
    for (int k = 1; k <= Lmax; k++) {
        T W = 0, WX = 0, WY = 0;
        for (int t = 0; t < m; t++) {
            int u = t + 1 == m ? 0 : t + 1;
            level_sum<T>(V, xi, yi, vx[t], vy[t], vx[u], vy[u], k - 1, W, WX, WY);
        }
        if (!(W > 0)) return;
        T iW = (T)1 / W;
        T ccx = WX * iW, ccy = WY * iW;
        T dx = ccx - px, dy = ccy - py;
        bool conv = dx * dx + dy * dy < E * E;
        if (conv || k == Lmax) {
            cx = xi + ccx;
            cy = yi + ccy;
            level = k;
            capped = !conv;
            return;
        }
        px = ccx;
        py = ccy;
    }
}

// ------------------------------------------------------------------ update
// one block per chunk of kThreads slots (one mesh in a batch).  MV selects the
// move the variant computes (0 DistMesh, 1 CVD); both variants are launched
// and the one that does not match the mesh's move of this iteration returns at
// once, so each is compiled (and register-allocated) for its own move.
template <typename T, bool B, int MV>
__global__ void __launch_bounds__(kThreads) k_update(const __grid_constant__ IterArgs<T> a) {
    const MeshView& V = mesh_of<B>(a, blockIdx.x * kThreads);
    if (V.ctrl->terminated || (V.ctrl->method_now != 0) != (MV != 0)) return;
    const DevParams& P = V.P;
    // a DistMesh iteration that keeps the last triangulation moves the current
    // state (copied to wrk); otherwise the state sorted at the triangulation
    const bool keep = !V.ctrl->retri;
    const T* IX = keep ? a.wrk.x : a.srt.x;
    const T* IY = keep ? a.wrk.y : a.srt.y;
    const bool track = P.fac_retria > 0.0 && V.ctrl->method_param == 0;
    unsigned moved = 0;
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    float devf = 0.f;  // size deviation summed over the owned valid edges
    int nown = 0, notsmall = 0;
    unsigned long long nfail = 0, tcap = 0, qcap = 0;
    if (s < a.n && (!B || s - V.soff < V.n)) {
        T xi = IX[s], yi = IY[s];
        int idi = a.srt.id[s];
        int ocls = keep ? a.wrk.cls[s] : a.srt.cls[s];
        T dprev = keep ? a.wrk.dprev[s] : a.srt.dprev[s];
        T h = (T)V.gh[a.cell[s]];
        int ne = a.ring_n[s];
        uint64_t vm = a.vmask[s];
        int lab[kRingCap];
        const int4* row = reinterpret_cast<const int4*>(a.ring + (size_t)s * kRingCap);
        for (int q = 0; q < (ne + 3) / 4; q++) {
            int4 v = row[q];
            lab[4 * q] = v.x;
            lab[4 * q + 1] = v.y;
            lab[4 * q + 2] = v.z;
            lab[4 * q + 3] = v.w;
        }
        T fac_mu = (T)V.ctrl->fac_mu;
        T Fx = 0, Fy = 0, fs = 0;
        // DistMesh forces on the valid edges (Eqs. 2-3); also the size deviation
        // (a float statistic; in CVD iterations it is all this loop computes)
        const float4 pi4 = a.pf[s];
        // FP64 mode: the sizing at each edge midpoint in float-float, from the
        // float-pair positions of the triangulation or split from the current
        // ones (iterations that keep the triangulation)
        ff fxi{pi4.x, pi4.y}, fyi{pi4.z, pi4.w};
        if (sizeof(T) == 8 && keep) {
            fxi = ff_from_d((double)xi);
            fyi = ff_from_d((double)yi);
        }
        const T l0f = (T)P.fac_F * fac_mu;
        // FP64 mode with the triangulation's positions: the whole spring sum in
        // float-float, from positions held exactly as three floats
        const bool ffs = sizeof(T) == 8 && !keep;
        const float2 pi3 = ffs ? a.pf3[s] : make_float2(0.f, 0.f);
        const ff l0ff = ffs ? ff_from_d((double)l0f) : ff{0.f, 0.f};
        const ff kff = ffs ? ff_from_d(P.k_spring) : ff{0.f, 0.f};
        ff FxF{0.f, 0.f}, FyF{0.f, 0.f}, fsF{0.f, 0.f};
        for (int t = 0; t < ne; t++) {
            int j = lab[t];
            if (j < 0) continue;
            int tp = t == 0 ? ne - 1 : t - 1;
            if (!((vm >> t) & 1ull) && !((vm >> tp) & 1ull)) continue;
            bool owner = idi < a.srt.id[j];
            if constexpr (MV != 0) {
                if (owner) {
                    float4 pj4 = a.pf[j];
                    float ex = ff_diff(pi4.x, pi4.y, pj4.x, pj4.y), ey = ff_diff(pi4.z, pi4.w, pj4.z, pj4.w);
                    float muf = bilin<float>(V.siz, pj4.x + 0.5f * ex, pj4.z + 0.5f * ey);
                    devf += fabsf(sqrtf(ex * ex + ey * ey) / ((float)fac_mu * muf) - 1.0f);
                    nown++;
                }
                continue;
            }
            if (ffs) {
                float4 pj4 = a.pf[j];
                float2 pj3 = a.pf3[j];
                ff dx = ff_diff3(pi4.x, pi4.y, pi3.x, pj4.x, pj4.y, pj3.x);
                ff dy = ff_diff3(pi4.z, pi4.w, pi3.y, pj4.z, pj4.w, pj3.y);
                ff l2 = ff_add(ff_mul(dx, dx), ff_mul(dy, dy));
                ff r = ff_rsqrt(l2);
                ff l = ff_mul(l2, r);
                ff mu = bilin_ff(V.siz, ff_scale2(ff_add(fxi, ff{pj4.x, pj4.y}), 0.5f),
                                 ff_scale2(ff_add(fyi, ff{pj4.z, pj4.w}), 0.5f));
                if (owner) {
                    devf += fabsf(l.h / ((float)fac_mu * mu.h) - 1.0f);
                    nown++;
                }
                ff l0 = ff_mul(l0ff, mu);
                if (ff_gt(l0, l)) {
                    ff fl = ff_mul(kff, ff_add_f(ff_mul(l0, r), -1.0f));  // f / l with f = k (l0 - l)
                    FxF = ff_add(FxF, ff_mul(fl, dx));
                    FyF = ff_add(FyF, ff_mul(fl, dy));
                    fsF = ff_add(fsF, ff_mul(kff, ff_sub(l0, l)));
                }
                continue;
            }
            T xj = IX[j], yj = IY[j];
            T dx = xi - xj, dy = yi - yj;
            T l2 = dx * dx + dy * dy;
            T r = rsqrt(l2);  // 1 / l: one reciprocal square root instead of a root and a division
            T l = l2 * r;
            T mu;
            float muf;
            if (sizeof(T) == 8) {
                ff fxj, fyj;
                if (keep) {
                    fxj = ff_from_d((double)xj);
                    fyj = ff_from_d((double)yj);
                } else {
                    float4 pj4 = a.pf[j];
                    fxj = ff{pj4.x, pj4.y};
                    fyj = ff{pj4.z, pj4.w};
                }
                ff m = bilin_ff(V.siz, ff_scale2(ff_add(fxi, fxj), 0.5f), ff_scale2(ff_add(fyi, fyj), 0.5f));
                mu = (T)ff_to_d(m);
                muf = m.h;
            } else {
                // FP32 mode: the midpoint (exact as a float pair) and the
                // lookup's grid coordinate in float-float, so mu carries one
                // rounding; a float midpoint and coordinate perturb mu by up to
                // |grad mu| |m| 2^-22, several 1e-6 of the smallest sizes here
                ff m = bilin_ff(V.siz, ff_scale2(two_sum((float)xi, (float)xj), 0.5f),
                                ff_scale2(two_sum((float)yi, (float)yj), 0.5f));
                mu = (T)m.h;
                muf = m.h;
            }
            if (owner) {
                devf += fabsf((float)l / ((float)fac_mu * muf) - 1.0f);
                nown++;
            }
            T l0 = l0f * mu;
            if (l < l0) {
                T k = (T)P.k_spring;
                T fl = k * (l0 * r - (T)1);  // f / l with f = k (l0 - l)
                Fx += fl * dx;
                Fy += fl * dy;
                fs += k * (l0 - l);
            }
        }
        if (ffs) {
            Fx = (T)ff_to_d(FxF);
            Fy = (T)ff_to_d(FyF);
            fs = (T)ff_to_d(fsF);
        }
        T pnx, pny, cx = xi, cy = yi;
        int qlv = 0;
        if constexpr (MV == 0) {
            pnx = xi + (T)P.dt * Fx;  // forward Euler (Eq. 5)
            pny = yi + (T)P.dt * Fy;
        } else {
            bool capped;
            cvd_centroid<T>(a, V, s, ne, lab, xi, yi, h, dprev, cx, cy, qlv, capped);
            if (capped) qcap++;
            pnx = cx;
            pny = cy;
        }
        // Sec. 4.3: clamp, classify, project
        T fx, fy;
        int ncls;
        treat_move<T>(V, xi, yi, ocls, pnx, pny, (T)P.fac_pt * h, fx, fy, ncls, tcap, nfail);
        if (track) {
            // Algorithm 1: distance from the position at the last triangulation
            T ex = fx - a.srt.x[s], ey = fy - a.srt.y[s];
            if (sqrt(ex * ex + ey * ey) > (T)P.fac_retria * h) moved = 1;
        }
        T mvx = fx - xi, mvy = fy - yi;
        T mv = sqrt(mvx * mvx + mvy * mvy);
        if (ocls == PT_INNER && !(mv < (T)P.fac_end * h)) notsmall = 1;
        a.cur.x[s] = fx;
        a.cur.y[s] = fy;
        a.cur.id[s] = idi;
        a.cur.cls[s] = (uint8_t)ncls;
        a.cur.dprev[s] = mv;
        if (P.debug) {
            size_t n = (size_t)a.n, id = (size_t)idi;
            a.dbg[2 * id] = (double)pnx;
            a.dbg[2 * id + 1] = (double)pny;
            a.dbg[2 * n + 2 * id] = (double)Fx;
            a.dbg[2 * n + 2 * id + 1] = (double)Fy;
            a.dbg[4 * n + 2 * id] = (double)cx;
            a.dbg[4 * n + 2 * id + 1] = (double)cy;
            a.dbg[6 * n + id] = (double)fs;
            a.dbg[7 * n + id] = (double)ncls;
            a.dbg[8 * n + id] = (double)mv;
            a.dbg[9 * n + id] = (double)qlv;
        }
    }
    if (__any_sync(0xffffffffu, moved) && (threadIdx.x & 31) == 0) V.ctrl->moved_far = 1;
    unsigned m = __ballot_sync(0xffffffffu, nfail != 0);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&V.ctrl->cnt.newton_fail, (unsigned long long)__popc(m));
    m = __ballot_sync(0xffffffffu, tcap != 0);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&V.ctrl->cnt.trace_cap, (unsigned long long)__popc(m));
    m = __ballot_sync(0xffffffffu, qcap != 0);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&V.ctrl->cnt.quad_cap, (unsigned long long)__popc(m));
    // block sums: the deviation in float-float and the counts as integers
    // within each warp, in double across the warps
    ff dv = warp_sum_ff(ff{devf, 0.f});
    int ne_w = __reduce_add_sync(0xffffffffu, nown), ns_w = __reduce_or_sync(0xffffffffu, notsmall);
    __shared__ double sh[3][kThreads / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][w] = ff_to_d(dv);
        sh[1][w] = (double)ne_w;
        sh[2][w] = (double)ns_w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double v0 = 0, v1 = 0, v2 = 0;
        for (int k = 0; k < kThreads / 32; k++) {
            v0 += sh[0][k];
            v1 += sh[1][k];
            v2 += sh[2][k];
        }
        a.up[blockIdx.x].size_dev = v0;
        a.up[blockIdx.x].n_edge = v1;
        a.up[blockIdx.x].not_small = v2;
    }
}

template <typename T>
void launch_update(const IterArgs<T>& a, int nblocks, cudaStream_t st) {
    if (a.Vs) {
        k_update<T, true, 0><<<nblocks, kThreads, 0, st>>>(a);
        k_update<T, true, 1><<<nblocks, kThreads, 0, st>>>(a);
    } else {
        k_update<T, false, 0><<<nblocks, kThreads, 0, st>>>(a);
        k_update<T, false, 1><<<nblocks, kThreads, 0, st>>>(a);
    }
}
template void launch_update<double>(const IterArgs<double>&, int, cudaStream_t);
template void launch_update<float>(const IterArgs<float>&, int, cudaStream_t);

// ------------------------------------------------------------------ statistics
constexpr int kStatThreads = 512;

// one block per mesh: reduces the mesh's emit partials [c0, c1)
template <typename T, bool B>
__global__ void __launch_bounds__(kStatThreads) k_stats_pre(const __grid_constant__ IterArgs<T> a, int decide) {
    const MeshView& V = B ? a.Vs[blockIdx.x] : a.V;
    DevCtrl* ctrl = V.ctrl;
    const DevParams& P = V.P;
    const EmitPartial* ep = a.ep;
    if (!a.force && ctrl->terminated) return;
    double acc[9] = {0, 0, 0, 0, 0, 180.0, 0, 0, 0};
    for (int b = V.c0 + threadIdx.x; b < V.c1; b += blockDim.x) {
        const double* p = reinterpret_cast<const double*>(&ep[b]);
        for (int q = 0; q < 9; q++)
            acc[q] = (q == 3 || q == 4) ? fmax(acc[q], p[q]) : (q == 5 ? fmin(acc[q], p[q]) : acc[q] + p[q]);
    }
    __shared__ double sh[kStatThreads][9];
    for (int q = 0; q < 9; q++) sh[threadIdx.x][q] = acc[q];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 9; q++) {
                double o = sh[threadIdx.x + w][q];
                sh[threadIdx.x][q] = (q == 3 || q == 4) ? fmax(sh[threadIdx.x][q], o)
                                   : (q == 5 ? fmin(sh[threadIdx.x][q], o) : sh[threadIdx.x][q] + o);
            }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double n = sh[0][0];
    double qa = n > 0 ? (sh[0][1] / n) * (sh[0][1] / n) : 0.0;
    double qb = n > 0 ? (sh[0][2] / n) * (sh[0][2] / n) : 0.0;
    double qm = sh[0][3];
    if (!a.force && !ctrl->retri) {
        // the iteration keeps the last triangulation: only fac_mu (Eq. 3, at
        // the current positions) changes; no quality, no decision
        ctrl->fac_mu = sh[0][6] > 0 ? sqrt(sh[0][7] / sh[0][8]) : 1.0;
        ctrl->method_now = 0;
        ctrl->last_method = 0;
        ctrl->iterations += 1;
        return;
    }
    if (decide) ctrl->cnt.triangulations += 1;
    ctrl->n_tri = n;
    ctrl->half_a = qa;
    ctrl->half_b = qb;
    ctrl->max_a = qm;
    ctrl->max_b = sh[0][4];
    ctrl->min_ang = n > 0 ? sh[0][5] : 0.0;
    ctrl->n_edges = sh[0][6];
    ctrl->fac_mu = sh[0][6] > 0 ? sqrt(sh[0][7] / sh[0][8]) : 1.0;
    if (!decide) return;
    double ra = 1, rb = 1, rm = 1;
    if (ctrl->have_prev) {
        ra = ctrl->prev_a > 0 ? fabs(qa - ctrl->prev_a) / ctrl->prev_a : 1.0;
        rb = ctrl->prev_b > 0 ? fabs(qb - ctrl->prev_b) / ctrl->prev_b : 1.0;
        rm = ctrl->prev_amax > 0 ? fabs(qm - ctrl->prev_amax) / ctrl->prev_amax : 1.0;
    }
    bool qend = ctrl->have_prev && ra < P.T_end_q && rb < P.T_end_q && rm < P.T_end_amax;
    int method, term = 0;
    if (P.adding) {
        // Sec. 3.6: until N_total is reached a stalled mesh gets new points
        // (the host adds them while the graph is paused: terminated = 2);
        // the hybrid switch and the termination tests wait for N_total
        if (ctrl->have_prev && ra < P.T_add && rb < P.T_add && n > 0) {
            ctrl->have_prev = 0;  // the next change is not measured across the addition
            ctrl->iterations += 1;
            ctrl->terminated = 2;
            return;
        }
        method = ctrl->method_param == 1 ? 1 : 0;
    } else if (ctrl->method_param == 2) {
        if (!ctrl->switched) {
            if (ctrl->have_prev && ra < P.T_switch) ctrl->switched = 1;  // Sec. 4.2
        } else if (qend) {
            term = 1;
        }
        method = ctrl->switched ? 1 : 0;
    } else {
        method = ctrl->method_param;
        term = qend;
    }
    if (ctrl->target_min_ang > 0.0 && !P.adding) {
        // a quality target replaces the quality termination test: iterate
        // until the minimum angle reaches it
        term = n > 0 && ctrl->min_ang >= ctrl->target_min_ang;
        if (term) ctrl->target_reached = 1;
    }
    ctrl->prev_a = qa;
    ctrl->prev_b = qb;
    ctrl->prev_amax = qm;
    ctrl->have_prev = 1;
    ctrl->method_now = method;
    ctrl->iterations += 1;
    if (term) ctrl->terminated = 1;
    else ctrl->last_method = method;
}

template <typename T, bool B>
__global__ void __launch_bounds__(kStatThreads) k_stats_post(const __grid_constant__ IterArgs<T> a) {
    const MeshView& V = B ? a.Vs[blockIdx.x] : a.V;
    DevCtrl* ctrl = V.ctrl;
    const UpdatePartial* up = a.up;
    if (ctrl->terminated) return;
    double acc[3] = {0, 0, 0};
    for (int b = V.c0 + threadIdx.x; b < V.c1; b += blockDim.x) {
        acc[0] += up[b].size_dev;
        acc[1] += up[b].n_edge;
        acc[2] += up[b].not_small;
    }
    __shared__ double sh[kStatThreads][3];
    for (int q = 0; q < 3; q++) sh[threadIdx.x][q] = acc[q];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 3; q++) sh[threadIdx.x][q] += sh[threadIdx.x + w][q];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    ctrl->size_dev = sh[0][1] > 0 ? sh[0][0] / sh[0][1] : 0.0;
    int small = sh[0][2] == 0.0;
    ctrl->small_moves = small;
    if (small && !V.P.adding) ctrl->terminated = 1;  // Sec. 4: every inner move below fac_end * h_i
    // Algorithm 1: DistMesh re-triangulates after a large movement only
    ctrl->retri = ctrl->method_param != 0 || !(V.P.fac_retria > 0.0) || ctrl->moved_far;
    ctrl->moved_far = 0;
}

template <typename T>
void launch_stats_pre(const IterArgs<T>& a, int decide, cudaStream_t st) {
    if (a.Vs) k_stats_pre<T, true><<<a.nmesh, kStatThreads, 0, st>>>(a, decide);
    else k_stats_pre<T, false><<<1, kStatThreads, 0, st>>>(a, decide);
}
template <typename T>
void launch_stats_post(const IterArgs<T>& a, cudaStream_t st) {
    if (a.Vs) k_stats_post<T, true><<<a.nmesh, kStatThreads, 0, st>>>(a);
    else k_stats_post<T, false><<<1, kStatThreads, 0, st>>>(a);
}
template void launch_stats_pre<double>(const IterArgs<double>&, int, cudaStream_t);
template void launch_stats_pre<float>(const IterArgs<float>&, int, cudaStream_t);
template void launch_stats_post<double>(const IterArgs<double>&, cudaStream_t);
template void launch_stats_post<float>(const IterArgs<float>&, cudaStream_t);

}  // namespace trime
