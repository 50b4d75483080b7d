// treat.cuh -- point treatment after a move (TriMe++ Sec. 4.3): clamp the
// move, classify the new position on the geometry grid, and bring an escaped
// point back by sphere tracing (from an inner point) or damped Newton
// projection (from a boundary point, Eqs. 8-10).  Shared by the iteration's
// update kernel and the learned proposal.
#pragma once
#include "kernels.cuh"

namespace trime {

// ------------------------------------------------------------------ point treatment
template <typename T>
__device__ __forceinline__ T geps_at(const MeshView& V, T x, T y) {
    int gi, gj;
    point_cell_t<T>(V.sdf, x, y, gi, gj);
    return (T)V.ggeps[gj * (V.sdf.nx - 1) + gi];
}

template <typename T>
__device__ int classify(const MeshView& V, T x, T y) {
    int gi, gj;
    if (!point_cell_t<T>(V.sdf, x, y, gi, gj)) return PT_OUTSIDE;
    int c = gj * (V.sdf.nx - 1) + gi;
    uint8_t k = V.gcls[c];
    if (k == CELL_OUTER) return PT_OUTSIDE;
    if (k == CELL_INNER) return PT_INNER;
    T s = bilin<T>(V.sdf, x, y), g = (T)V.ggeps[c];
    if (fabs(s) <= g) return PT_BOUNDARY;
    if (s < -g) return PT_INNER;
    return PT_OUTSIDE;
}

// sphere tracing from an inner p_old toward an outside p_new (Fig. 21a)
template <typename T>
__device__ bool sphere_trace(const MeshView& V, T ax, T ay, T bx, T by, T& ox, T& oy) {
    T Lx = bx - ax, Ly = by - ay;
    T L = sqrt(Lx * Lx + Ly * Ly);
    T ux = Lx / L, uy = Ly / L;
    T x = ax, y = ay, lox = ax, loy = ay, hix = bx, hiy = by, t = 0;
    int it = 0;
    bool bisect = false;
    for (; it < V.P.trace_max; it++) {
        T s = bilin<T>(V.sdf, x, y), g = geps_at(V, x, y);
        if (fabs(s) <= g) { ox = x; oy = y; return false; }
        if (s > g) { hix = x; hiy = y; bisect = true; break; }
        lox = x; loy = y;
        t += fabs(s);
        if (t >= L) { bisect = true; break; }
        x = ax + t * ux;
        y = ay + t * uy;
    }
    if (bisect)
        for (it++; it < V.P.trace_max; it++) {
            T mx = (lox + hix) * (T)0.5, my = (loy + hiy) * (T)0.5;
            T s = bilin<T>(V.sdf, mx, my), g = geps_at(V, mx, my);
            if (fabs(s) <= g) { ox = mx; oy = my; return false; }
            if (s < 0) { lox = mx; loy = my; } else { hix = mx; hiy = my; }
        }
    ox = lox;
    oy = loy;
    return true;
}

// damped Newton projection (Eqs. 8-10), gradient at the iterate, exact
// derivatives of the bilinear interpolant
template <typename T>
__device__ void newton_project(const MeshView& V, T pnx, T pny, T& ox, T& oy) {
    T x = pnx, y = pny;
    for (int k = 0; k < V.P.newton_max; k++) {
        T f, fx, fy, fxy;
        bilin_grad<T>(V.sdf, x, y, f, fx, fy, fxy);
        T L1 = f;
        T L2 = (x - pnx) * fy - (y - pny) * fx;
        T J00 = fx, J01 = fy;
        T J10 = fy + (x - pnx) * fxy, J11 = -fx - (y - pny) * fxy;
        T det = J00 * J11 - J01 * J10;
        if (det == (T)0 || !isfinite(det)) break;
        T dx = (J11 * L1 - J01 * L2) / det;
        T dy = (-J10 * L1 + J00 * L2) / det;
        x -= (T)V.P.damping * dx;
        y -= (T)V.P.damping * dy;
        if (fabs(bilin<T>(V.sdf, x, y)) <= geps_at(V, x, y)) break;
    }
    ox = x;
    oy = y;
}

// clamp the raw move p -> pn to length Tm, classify, project; returns the
// treated position and class (Sec. 4.3); counts trace caps and Newton failures
template <typename T>
__device__ __forceinline__ void treat_move(const MeshView& V, T xi, T yi, int ocls, T pnx, T pny, T Tm, T& fx,
                                           T& fy, int& ncls, unsigned long long& tcap,
                                           unsigned long long& nfail) {
    T dx = pnx - xi, dy = pny - yi;
    T d = sqrt(dx * dx + dy * dy);
    T qx = pnx, qy = pny;
    if (d > Tm) {
        qx = xi + dx * (Tm / d);
        qy = yi + dy * (Tm / d);
    }
    int c = classify(V, qx, qy);
    fx = qx;
    fy = qy;
    ncls = c;
    if (c == PT_OUTSIDE) {
        T ox, oy;
        if (ocls == PT_INNER) {
            if (sphere_trace(V, xi, yi, qx, qy, ox, oy)) tcap++;
            int cc = classify(V, ox, oy);
            if (cc == PT_OUTSIDE) { fx = xi; fy = yi; ncls = ocls; }
            else { fx = ox; fy = oy; ncls = cc; }
        } else {
            newton_project(V, qx, qy, ox, oy);
            if (classify(V, ox, oy) == PT_BOUNDARY) { fx = ox; fy = oy; ncls = PT_BOUNDARY; }
            else { nfail++; fx = xi; fy = yi; ncls = ocls; }
        }
    }
}

}  // namespace trime
