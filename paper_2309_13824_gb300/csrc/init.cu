// init.cu -- initial points of TriMe++ Sec. 3.5 on the device: the k-th point
// is uniform in its (dithered) cell by the counter-based SplitMix64 stream,
// and a point of a boundary cell whose SDF exceeds that cell's geps is
// projected onto the boundary by the damped Newton iteration of Sec. 4.3,
// written with fixed FP64 operations so every point is reproducible bit for
// bit.
#include "kernels.cuh"

namespace trime {

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t n) {
    uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// value and exact derivatives of the bilinear interpolant, fixed formulas
__device__ __forceinline__ void bilin_d_fixed(const DevGrid& g, double x, double y, double& f, double& fx_,
                                              double& fy_, double& fxy) {
    int i, j;
    double fx, fy;
    grid_locate(g, x, y, i, j, fx, fy);
    const float* r0 = g.v + (size_t)j * g.nx + i;
    const float* r1 = r0 + g.nx;
    double v00 = r0[0], v10 = r0[1], v01 = r1[0], v11 = r1[1];
    double a = fadd(v00, fmul(fx, fsub(v10, v00)));
    double b = fadd(v01, fmul(fx, fsub(v11, v01)));
    f = fadd(a, fmul(fy, fsub(b, a)));
    double d0 = fsub(v10, v00), d1 = fsub(v11, v01);
    fx_ = fdiv(fadd(d0, fmul(fy, fsub(d1, d0))), g.dx);
    fy_ = fdiv(fsub(b, a), g.dy);
    fxy = fdiv(fsub(d1, d0), fmul(g.dx, g.dy));
}

__global__ void k_init_points(const DevGrid sdf, const uint8_t* gcls, const double* ggeps, const int32_t* pcell,
                              int64_t n, uint64_t seed, double damping, int newton_max, double* out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    int ncx = sdf.nx - 1;
    int c = pcell[q], gi = c % ncx, gj = c / ncx;
    double u = (double)(splitmix64(seed, (uint64_t)(2 * q)) >> 11) * 0x1.0p-53;
    double w = (double)(splitmix64(seed, (uint64_t)(2 * q + 1)) >> 11) * 0x1.0p-53;
    double cx0 = fadd(sdf.x0, fmul((double)gi, sdf.dx)), cy0 = fadd(sdf.y0, fmul((double)gj, sdf.dy));
    double x = fadd(cx0, fmul(u, sdf.dx)), y = fadd(cy0, fmul(w, sdf.dy));
    if (gcls[c] == CELL_BOUNDARY && bilin_fixed(sdf, x, y) > ggeps[c]) {
        // damped Newton projection (Eqs. 8-10), gradient at the iterate; it
        // counts only when it ends as a boundary point (Sec. 4.3 classes)
        double x0 = x, y0 = y;
        double pnx = x, pny = y;
        for (int k = 0; k < newton_max; k++) {
            double f, fx, fy, fxy;
            bilin_d_fixed(sdf, x, y, f, fx, fy, fxy);
            double ex = fsub(x, pnx), ey = fsub(y, pny);
            double L1 = f;
            double L2 = fsub(fmul(ex, fy), fmul(ey, fx));
            double J00 = fx, J01 = fy;
            double J10 = fadd(fy, fmul(ex, fxy)), J11 = fsub(-fx, fmul(ey, fxy));
            double det = fsub(fmul(J00, J11), fmul(J01, J10));
            if (det == 0.0 || !isfinite(det)) break;
            double dx = fdiv(fsub(fmul(J11, L1), fmul(J01, L2)), det);
            double dy = fdiv(fadd(fmul(-J10, L1), fmul(J00, L2)), det);
            x = fsub(x, fmul(damping, dx));
            y = fsub(y, fmul(damping, dy));
            int ci, cj;
            point_cell_fixed(sdf, x, y, ci, cj);
            if (fabs(bilin_fixed(sdf, x, y)) <= ggeps[cj * ncx + ci]) break;
        }
        int ci, cj;
        bool on = point_cell_fixed(sdf, x, y, ci, cj) && gcls[cj * ncx + ci] == CELL_BOUNDARY &&
                  fabs(bilin_fixed(sdf, x, y)) <= ggeps[cj * ncx + ci];
        if (!on) {
            x = x0;
            y = y0;
        }
    }
    out[2 * q] = x;
    out[2 * q + 1] = y;
}

void launch_init_points(const DevGrid& sdf, const uint8_t* gcls, const double* ggeps, const int32_t* pcell,
                        int64_t n, uint64_t seed, double damping, int newton_max, double* out, cudaStream_t st) {
    if (n <= 0) return;
    k_init_points<<<(int)((n + 255) / 256), 256, 0, st>>>(sdf, gcls, ggeps, pcell, n, seed, damping, newton_max,
                                                          out);
}

}  // namespace trime
