// exact.cuh -- exact incircle / orientation signs on the device.
//
// Floating-point expansion arithmetic after Shewchuk, "Adaptive Precision
// Floating-Point Arithmetic and Fast Robust Geometric Predicates" (1997):
// a value is a sum of non-overlapping doubles; sums use two-sum, products use
// the exact fused-multiply-add product error.  Results are compressed after
// every product so the fixed-capacity buffers stay short.  Exact ties are
// broken by symbolic perturbation of the lifted coordinate: point r's lift is
// |p_r|^2 + eps^(id_r + 1), so smaller ids carry larger perturbations.
//
// Guard: the arithmetic is exact while every non-zero coordinate difference
// lies in [1e-50, 1e50] (no underflow of product error terms) and expansions
// fit kExpCap components; otherwise the predicates return kExactFail.
#pragma once
#include "common.cuh"

namespace trime {

constexpr int kExpCap = 48;

__device__ __forceinline__ void two_sum(double a, double b, double& x, double& y) {
    x = __dadd_rn(a, b);
    double bv = __dsub_rn(x, a);
    double av = __dsub_rn(x, bv);
    double br = __dsub_rn(b, bv);
    double ar = __dsub_rn(a, av);
    y = __dadd_rn(ar, br);
}

__device__ __forceinline__ void fast_two_sum(double a, double b, double& x, double& y) {
    x = __dadd_rn(a, b);
    double bv = __dsub_rn(x, a);
    y = __dsub_rn(b, bv);
}

__device__ __forceinline__ void two_diff(double a, double b, double& x, double& y) {
    x = __dsub_rn(a, b);
    double bv = __dsub_rn(a, x);
    double av = __dadd_rn(x, bv);
    double br = __dsub_rn(bv, b);
    double ar = __dsub_rn(a, av);
    y = __dadd_rn(ar, br);
}

__device__ __forceinline__ void two_prod(double a, double b, double& x, double& y) {
    x = __dmul_rn(a, b);
    y = __fma_rn(a, b, -x);
}

// h = e + b (zero-eliminating); returns length or -1 on overflow
__device__ __forceinline__ int grow_expansion(int elen, const double* e, double b, double* h, int cap) {
    double Q = b;
    int hl = 0;
    for (int i = 0; i < elen; i++) {
        double Qn, hh;
        two_sum(Q, e[i], Qn, hh);
        Q = Qn;
        if (hh != 0.0) {
            if (hl >= cap) return -1;
            h[hl++] = hh;
        }
    }
    if (Q != 0.0 || hl == 0) {
        if (hl >= cap) return -1;
        h[hl++] = Q;
    }
    return hl;
}

// h = e + f by repeated growth (each step keeps the expansion non-overlapping)
__device__ __forceinline__ int expansion_sum(int elen, const double* e, int flen, const double* f, double* h, int cap) {
    double t[kExpCap];
    if (elen > kExpCap) return -1;
    for (int i = 0; i < elen; i++) t[i] = e[i];
    int tl = elen;
    for (int j = 0; j < flen; j++) {
        if (f[j] == 0.0) continue;
        tl = grow_expansion(tl, t, f[j], h, cap);
        if (tl < 0) return -1;
        for (int i = 0; i < tl; i++) t[i] = h[i];
    }
    for (int i = 0; i < tl; i++) h[i] = t[i];
    return tl;
}

// h = e * b (zero-eliminating)
__device__ __forceinline__ int scale_expansion(int elen, const double* e, double b, double* h, int cap) {
    double Q, hh;
    int hl = 0;
    two_prod(e[0], b, Q, hh);
    if (hh != 0.0) h[hl++] = hh;
    for (int i = 1; i < elen; i++) {
        double p1, p0, sum;
        two_prod(e[i], b, p1, p0);
        two_sum(Q, p0, sum, hh);
        if (hh != 0.0) {
            if (hl >= cap) return -1;
            h[hl++] = hh;
        }
        fast_two_sum(p1, sum, Q, hh);
        if (hh != 0.0) {
            if (hl >= cap) return -1;
            h[hl++] = hh;
        }
    }
    if (Q != 0.0 || hl == 0) {
        if (hl >= cap) return -1;
        h[hl++] = Q;
    }
    return hl;
}

// rewrite e (non-overlapping, increasing magnitude) with as few components as
// the two sweeps leave; in place
__device__ __forceinline__ int compress(int elen, double* e) {
    if (elen <= 1) return elen;
    double g[kExpCap];
    int bottom = elen - 1;
    double Q = e[bottom];
    for (int i = elen - 2; i >= 0; i--) {
        double Qn, q;
        fast_two_sum(Q, e[i], Qn, q);
        if (q != 0.0) {
            g[bottom--] = Qn;
            Q = q;
        } else {
            Q = Qn;
        }
    }
    g[bottom] = Q;
    int top = 0;
    for (int i = bottom + 1; i < elen; i++) {
        double Qn, q;
        fast_two_sum(g[i], Q, Qn, q);
        if (q != 0.0) e[top++] = q;
        Q = Qn;
    }
    e[top] = Q;
    return top + 1;
}

// h = e * f, compressed
__device__ __forceinline__ int expansion_mul(int elen, const double* e, int flen, const double* f, double* h, int cap) {
    double acc[kExpCap], t[kExpCap], s[kExpCap];
    int al = 1;
    acc[0] = 0.0;
    for (int j = 0; j < flen; j++) {
        int tl = scale_expansion(elen, e, f[j], t, kExpCap);
        if (tl < 0) return -1;
        al = expansion_sum(al, acc, tl, t, s, kExpCap);
        if (al < 0) return -1;
        al = compress(al, s);
        for (int i = 0; i < al; i++) acc[i] = s[i];
    }
    if (al > cap) return -1;
    for (int i = 0; i < al; i++) h[i] = acc[i];
    return al;
}

__device__ __forceinline__ int exp_sign(int len, const double* e) {
    for (int i = len - 1; i >= 0; i--)
        if (e[i] != 0.0) return e[i] > 0.0 ? 1 : -1;
    return 0;
}

__device__ __forceinline__ bool diff_ok(double a, double b) {
    double d = fabs(a - b);
    return d == 0.0 || (d >= 1e-50 && d <= 1e50);
}

// Status codes of the exact predicates: -1 / 0 / +1 are signs, kExactFail
// means the capacity or underflow guard tripped.
constexpr int kExactFail = 2;

// sign of (b-a) x (c-a), exact: the determinant with a column of ones is
// the sum of the six products ax by - ay bx + bx cy - by cx + cx ay - cy ax,
// each split exactly into two doubles and accumulated by growth
static __device__ __noinline__ int orient_exact(const double* a, const double* b, const double* c) {
    const double* P[3] = {a, b, c};
    bool ok = true;
    for (int k = 0; k < 3; k++)
        for (int q = 0; q < 2; q++) {
            double v = fabs(P[k][q]);
            ok = ok && (v == 0.0 || (v >= 1e-100 && v <= 1e100));
        }
    double acc[kExpCap], tmp[kExpCap];
    int al = 1;
    acc[0] = 0.0;
    for (int k = 0; k < 3 && ok; k++) {
        const double* u = P[k];
        const double* v = P[k == 2 ? 0 : k + 1];
        double t[4];
        two_prod(u[0], v[1], t[1], t[0]);
        two_prod(u[1], v[0], t[3], t[2]);
        t[2] = -t[2];
        t[3] = -t[3];
        for (int q = 0; q < 4 && ok; q++) {
            al = grow_expansion(al, acc, t[q], tmp, kExpCap);
            ok = al > 0;
            for (int i = 0; i < al; i++) acc[i] = tmp[i];
        }
    }
    return ok ? exp_sign(al, acc) : kExactFail;
}

// sign of det of rows [x, y, x^2 + y^2, 1] of (a, b, c, d), exact
static __device__ __noinline__ int incircle_exact(const double* a, const double* b, const double* c, const double* d) {
    const double* P[3] = {a, b, c};
    double dx[3][2], dy[3][2];
    bool ok = true;
    for (int r = 0; r < 3; r++) {
        ok = ok && diff_ok(P[r][0], d[0]) && diff_ok(P[r][1], d[1]);
        two_diff(P[r][0], d[0], dx[r][1], dx[r][0]);
        two_diff(P[r][1], d[1], dy[r][1], dy[r][0]);
    }
    double lift[3][kExpCap];
    int ll[3] = {0, 0, 0};
    double t1[kExpCap], t2[kExpCap];
    for (int r = 0; r < 3 && ok; r++) {
        int l1 = expansion_mul(2, dx[r], 2, dx[r], t1, kExpCap);
        int l2 = expansion_mul(2, dy[r], 2, dy[r], t2, kExpCap);
        ok = l1 > 0 && l2 > 0;
        if (ok) {
            ll[r] = expansion_sum(l1, t1, l2, t2, lift[r], kExpCap);
            ok = ll[r] > 0;
            if (ok) ll[r] = compress(ll[r], lift[r]);
        }
    }
    // det = lift_a (bx cy - by cx) + lift_b (cx ay - cy ax) + lift_c (ax by - ay bx)
    double acc[kExpCap];
    int al = 1;
    acc[0] = 0.0;
    for (int r = 0; r < 3 && ok; r++) {
        int u = (r + 1) % 3, v = (r + 2) % 3;
        double m[kExpCap], term[kExpCap], s[kExpCap];
        int l1 = expansion_mul(2, dx[u], 2, dy[v], t1, kExpCap);
        int l2 = expansion_mul(2, dy[u], 2, dx[v], t2, kExpCap);
        ok = l1 > 0 && l2 > 0;
        if (!ok) break;
        for (int i = 0; i < l2; i++) t2[i] = -t2[i];
        int ml = expansion_sum(l1, t1, l2, t2, m, kExpCap);
        ok = ml > 0;
        if (!ok) break;
        ml = compress(ml, m);
        int tl = expansion_mul(ll[r], lift[r], ml, m, term, kExpCap);
        ok = tl > 0;
        if (!ok) break;
        al = expansion_sum(al, acc, tl, term, s, kExpCap);
        ok = al > 0;
        if (!ok) break;
        al = compress(al, s);
        for (int i = 0; i < al; i++) acc[i] = s[i];
    }
    return ok ? exp_sign(al, acc) : kExactFail;
}

// Perturbed det4(a,b,c,d) sign (never 0 for the configurations used here):
// exact value first, then the coefficient of the largest perturbation with a
// non-zero cofactor: C_a = orient(b,c,d), C_b = -orient(a,c,d),
// C_c = orient(a,b,d), C_d = -orient(a,b,c).  Returns kExactFail on a guard.
static __device__ __noinline__ int incircle_sos(const double* a, int ia, const double* b, int ib, const double* c, int ic,
                                         const double* d, int id) {
    int s = incircle_exact(a, b, c, d);
    if (s == 0) {
        const double* P[4] = {a, b, c, d};
        int I[4] = {ia, ib, ic, id};
        int ord[4] = {0, 1, 2, 3};
        for (int x = 1; x < 4; x++)
            for (int y = x; y > 0 && I[ord[y]] < I[ord[y - 1]]; y--) {
                int t = ord[y];
                ord[y] = ord[y - 1];
                ord[y - 1] = t;
            }
        s = kExactFail;
        for (int q = 0; q < 4; q++) {
            int r = ord[q], cs;
            if (r == 0) cs = orient_exact(P[1], P[2], P[3]);
            else if (r == 1) cs = orient_exact(P[0], P[2], P[3]);
            else if (r == 2) cs = orient_exact(P[0], P[1], P[3]);
            else cs = orient_exact(P[0], P[1], P[2]);
            if (cs == kExactFail) break;
            if (r == 1 || r == 3) cs = -cs;
            if (cs != 0) {
                s = cs;
                break;
            }
        }
    }
    return s;
}

}  // namespace trime
