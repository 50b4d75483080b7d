// autosize.cu -- the automatic element sizing field of TriMe++ (App. A
// boundary samples, Sec. 3.3 medial axis and local feature size, Eq. 7).
//
// The serial steps (the sample trimming, whose result depends on its order,
// and the bookkeeping of the medial points) run on the host in native code
// with bucket grids; the data-parallel ones run on the device: the segment
// SDF grid, the Delaunay triangles of the samples (the meshing library's own
// Voronoi kernels, unbounded cells, no validity tests), the medial points
// read off them (k_medial) and the sizing field.  Every distance uses the
// same fixed FP64 formula as the definition (host code is built without
// FMA contraction), so the result is that definition's exactly.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "trime.h"

namespace {

constexpr double kFacS = 0.5;     // App. B fac_s
constexpr double kFacGeps = 0.01; // App. B fac_geps
constexpr double kFacNei = 2.0;   // App. B fac_nei
constexpr int kNThres = 3;        // App. B n_nei^thres

double dist(double ax, double ay, double bx, double by) {
    double dx = bx - ax, dy = by - ay;
    return std::sqrt(dx * dx + dy * dy);
}

// distance from (x, y) to the closest segment of the loop
double seg_min_dist(const double* xy, int64_t nv, double x, double y) {
    double best = INFINITY;
    for (int64_t k = 0; k < nv; k++) {
        int64_t k1 = k + 1 == nv ? 0 : k + 1;
        double ax = xy[2 * k], ay = xy[2 * k + 1];
        double ex = xy[2 * k1] - ax, ey = xy[2 * k1 + 1] - ay;
        double wx = x - ax, wy = y - ay;
        double t = (wx * ex + wy * ey) / (ex * ex + ey * ey);
        if (!(t > 0.0)) t = 0.0;
        if (t > 1.0) t = 1.0;
        double cx = ax + t * ex, cy = ay + t * ey;
        double dx = x - cx, dy = y - cy;
        double d = std::sqrt(dx * dx + dy * dy);
        if (d < best) best = d;
    }
    return best;
}

// a uniform bucket grid of points that can move and disappear
struct Buckets {
    double x0, y0, bs;
    int gx, gy;
    std::vector<std::vector<int32_t>> b;
    void init(double ax, double ay, double bx, double by, double size, int64_t maxb) {
        double W = std::max(bx - ax, size), H = std::max(by - ay, size);
        bs = std::max(size, std::sqrt(W * H / (double)maxb));
        x0 = ax;
        y0 = ay;
        gx = std::max(1, (int)std::ceil(W / bs) + 1);
        gy = std::max(1, (int)std::ceil(H / bs) + 1);
        b.assign((size_t)gx * gy, {});
    }
    int ix(double x) const { return std::min(gx - 1, std::max(0, (int)std::floor((x - x0) / bs))); }
    int iy(double y) const { return std::min(gy - 1, std::max(0, (int)std::floor((y - y0) / bs))); }
    std::vector<int32_t>& at(double x, double y) { return b[(size_t)iy(y) * gx + ix(x)]; }
    void insert(int32_t i, double x, double y) { at(x, y).push_back(i); }
    void erase(int32_t i, double x, double y) {
        auto& v = at(x, y);
        v.erase(std::find(v.begin(), v.end(), i));
    }
    // distance from (x, y) to the outside of the block of rings 0..r around (ci, cj)
    double outside(double x, double y, int ci, int cj, int r) const {
        double D = INFINITY;
        if (ci - r > 0) D = std::min(D, x - (x0 + (ci - r) * bs));
        if (ci + r < gx - 1) D = std::min(D, (x0 + (ci + r + 1) * bs) - x);
        if (cj - r > 0) D = std::min(D, y - (y0 + (cj - r) * bs));
        if (cj + r < gy - 1) D = std::min(D, (y0 + (cj + r + 1) * bs) - y);
        return D;
    }
    template <typename F>
    void ring(int ci, int cj, int r, F&& f) const {
        for (int j = cj - r; j <= cj + r; j++) {
            if (j < 0 || j >= gy) continue;
            int step = (j == cj - r || j == cj + r) ? 1 : 2 * r;
            for (int i = ci - r; i <= ci + r; i += step) {
                if (i < 0 || i >= gx) continue;
                for (int32_t q : b[(size_t)j * gx + i]) f(q);
            }
        }
    }
};

// App. A with segment input: the initial samples and the serial trimming
std::vector<double> boundary_samples(const double* xy, int64_t nv, double ds, double geps_hat) {
    std::vector<double> px, py;
    for (int64_t k = 0; k < nv; k++) {
        int64_t k1 = k + 1 == nv ? 0 : k + 1;
        double ax = xy[2 * k], ay = xy[2 * k + 1], ex = xy[2 * k1] - ax, ey = xy[2 * k1 + 1] - ay;
        double L = std::sqrt(ex * ex + ey * ey);
        px.push_back(ax);
        py.push_back(ay);
        if (L > ds) {
            int64_t m = (int64_t)std::floor(L / ds) + 1;
            for (int64_t q = 1; q < m; q++) {
                double t = (double)q / (double)m;
                px.push_back(ax + t * ex);
                py.push_back(ay + t * ey);
            }
        }
    }
    int64_t n = (int64_t)px.size();
    double bx0 = *std::min_element(px.begin(), px.end()), bx1 = *std::max_element(px.begin(), px.end());
    double by0 = *std::min_element(py.begin(), py.end()), by1 = *std::max_element(py.begin(), py.end());
    Buckets B;
    B.init(bx0, by0, bx1, by1, ds, (int64_t)1 << 22);
    for (int64_t i = 0; i < n; i++) B.insert((int32_t)i, px[i], py[i]);
    std::vector<uint8_t> alive(n, 1), done(n, 0);
    std::vector<std::pair<double, int32_t>> cand;
    bool any = true;
    while (any) {
        any = false;
        for (int64_t i = 0; i < n; i++) {
            if (!alive[i] || done[i]) continue;
            // the closest other point with a valid midpoint, in (distance, index) order
            int ci = B.ix(px[i]), cj = B.iy(py[i]);
            cand.clear();
            size_t next = 0;
            int32_t found = -1;
            double fd = 0.0, mx = 0.0, my = 0.0;
            for (int r = 0; found < 0; r++) {
                bool last = r > std::max(std::max(ci, B.gx - 1 - ci), std::max(cj, B.gy - 1 - cj));
                if (!last)
                    B.ring(ci, cj, r, [&](int32_t j) {
                        if (j != i) cand.emplace_back(dist(px[i], py[i], px[j], py[j]), j);
                    });
                std::sort(cand.begin() + next, cand.end());
                double D = last ? INFINITY : B.outside(px[i], py[i], ci, cj, r);
                while (next < cand.size() && (last || cand[next].first < D * (1.0 - 1e-12))) {
                    int32_t j = cand[next].second;
                    double cx = (px[i] + px[j]) * 0.5, cy = (py[i] + py[j]) * 0.5;
                    if (std::fabs(seg_min_dist(xy, nv, cx, cy)) <= geps_hat) {
                        found = j;
                        fd = cand[next].first;
                        mx = cx;
                        my = cy;
                        break;
                    }
                    next++;
                }
                if (last) break;
            }
            if (found < 0 || !(fd < ds)) {
                done[i] = 1;
                continue;
            }
            alive[found] = 0;
            B.erase(found, px[found], py[found]);
            B.erase((int32_t)i, px[i], py[i]);
            px[i] = mx;
            py[i] = my;
            B.insert((int32_t)i, px[i], py[i]);
            any = true;
        }
    }
    std::vector<double> out;
    for (int64_t i = 0; i < n; i++)
        if (alive[i]) {
            out.push_back(px[i]);
            out.push_back(py[i]);
        }
    return out;
}

// medial points with at least n_thres others within r_nei are kept (all if
// none would be); lfs of each sample = its distance to the closest kept one
int64_t local_feature_size(const std::vector<double>& S, const std::vector<double>& M, double r_nei,
                           std::vector<double>& lfs) {
    int64_t ns = (int64_t)S.size() / 2, nm = (int64_t)M.size() / 2;
    double ax = INFINITY, ay = INFINITY, bx = -INFINITY, by = -INFINITY;
    for (int64_t a = 0; a < nm; a++) {
        ax = std::min(ax, M[2 * a]);
        ay = std::min(ay, M[2 * a + 1]);
        bx = std::max(bx, M[2 * a]);
        by = std::max(by, M[2 * a + 1]);
    }
    Buckets B;
    B.init(ax, ay, bx, by, r_nei, (int64_t)1 << 22);
    for (int64_t a = 0; a < nm; a++) B.insert((int32_t)a, M[2 * a], M[2 * a + 1]);
    std::vector<uint8_t> keep(nm, 0);
    int64_t kept = 0;
    for (int64_t a = 0; a < nm; a++) {
        int c = 0;
        int ci = B.ix(M[2 * a]), cj = B.iy(M[2 * a + 1]);
        for (int r = 0; r <= 1; r++)
            B.ring(ci, cj, r, [&](int32_t b) {
                if (b != a && dist(M[2 * a], M[2 * a + 1], M[2 * b], M[2 * b + 1]) <= r_nei) c++;
            });
        keep[a] = c >= kNThres;
        kept += keep[a];
    }
    if (kept > 0) {
        Buckets K2;
        K2.init(ax, ay, bx, by, r_nei, (int64_t)1 << 22);
        for (int64_t a = 0; a < nm; a++)
            if (keep[a]) K2.insert((int32_t)a, M[2 * a], M[2 * a + 1]);
        B = std::move(K2);
    }
    lfs.assign(ns, INFINITY);
    for (int64_t i = 0; i < ns; i++) {
        double x = S[2 * i], y = S[2 * i + 1];
        int ci = B.ix(x), cj = B.iy(y);
        double best = INFINITY;
        int rmax = std::max(std::max(ci, B.gx - 1 - ci), std::max(cj, B.gy - 1 - cj));
        for (int r = 0; r <= rmax; r++) {
            B.ring(ci, cj, r, [&](int32_t a) { best = std::min(best, dist(x, y, M[2 * a], M[2 * a + 1])); });
            double D = B.outside(x, y, ci, cj, r);
            if (best < D * (1.0 - 1e-12)) break;
        }
        lfs[i] = best;
    }
    return kept;
}

}  // namespace

extern "C" int mesh_auto_sizing(const double* xy, int64_t nv, double K, double x0, double y0, double x1, double y1,
                                int32_t nx, int32_t ny, float* sdf_out, float* sizing_out, int64_t* counts,
                                void* cuda_stream) {
    using trime::set_error;
    if (!xy || !sizing_out) return set_error(TRIME_EINVAL, "NULL pointer");
    if (nv < 3) return set_error(TRIME_EINVAL, "need at least 3 vertices");
    if (nx < 2 || ny < 2 || !(x1 > x0) || !(y1 > y0)) return set_error(TRIME_EINVAL, "bad grid");
    if (!(K >= 0.0) || !std::isfinite(K)) return set_error(TRIME_EINVAL, "K must be finite and >= 0");
    double dx = (x1 - x0) / (double)(nx - 1), dy = (y1 - y0) / (double)(ny - 1);
    double g = std::min(dx, dy);
    double ds = kFacS * g, geps_hat = kFacGeps * g, r_nei = kFacNei * kNThres * ds;
    for (int64_t k = 0; k < 2 * nv; k++)
        if (!std::isfinite(xy[k])) return set_error(TRIME_EINVAL, "vertices must be finite");
    // the segment SDF grid (host copy: the meshing library deep-copies host grids)
    size_t nn = (size_t)nx * (size_t)ny;
    std::vector<float> sdf(nn);
    int rc = mesh_segment_sdf_grid(xy, nv, x0, y0, x1, y1, nx, ny, sdf.data(), cuda_stream);
    if (rc) return rc;
    // 1. boundary samples
    std::vector<double> S = boundary_samples(xy, nv, ds, geps_hat);
    int64_t ns = (int64_t)S.size() / 2;
    // 2. Delaunay triangles of the samples and their medial points
    mesh_params P;
    mesh_default_params(&P);
    P.bounded = 0;
    P.validity = 0;
    P.precision = 0;
    mesh_grid2d gs{nx, ny, x0, y0, x1, y1, sdf.data()};
    const float one[4] = {1.f, 1.f, 1.f, 1.f};
    mesh_grid2d gz{2, 2, x0, y0, x1, y1, one};
    mesh_t* m = nullptr;
    if ((rc = mesh_init(&m, &gs, &gz, S.data(), ns, &P, cuda_stream))) return rc;
    std::vector<double> v(4 * (size_t)ns);
    std::vector<uint8_t> fl((size_t)ns);
    mesh_stats st;
    rc = mesh_rebuild(m, &st);
    // cells with more edges than a ring row are a guard trip for the mesh but
    // are rebuilt in full for the medial points
    if (rc == TRIME_EDEVICE && st.exact_overflow == 0 && st.ring_overflow > 0) rc = TRIME_OK;
    if (!rc) rc = mesh_medial_points(m, v.data(), fl.data());
    mesh_destroy(m);
    if (rc) return rc;
    std::vector<double> M;
    for (int64_t i = 0; i < ns; i++) {
        if (fl[i] & 1) {
            M.push_back(v[4 * i]);
            M.push_back(v[4 * i + 1]);
        }
        if (fl[i] & 2) {
            M.push_back(v[4 * i + 2]);
            M.push_back(v[4 * i + 3]);
        }
    }
    if (M.empty()) return set_error(TRIME_EINVAL, "no medial points (degenerate shape)");
    // 3. trimmed medial points and lfs
    std::vector<double> lfs;
    int64_t kept = local_feature_size(S, M, r_nei, lfs);
    // 4. Eq. 7 on the grid
    if ((rc = mesh_sizing_field(S.data(), lfs.data(), ns, K, x0, y0, x1, y1, nx, ny, sizing_out, cuda_stream)))
        return rc;
    if (sdf_out) {
        cudaPointerAttributes at;
        bool dev = cudaPointerGetAttributes(&at, sdf_out) == cudaSuccess &&
                   (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
        cudaGetLastError();
        if (dev) {
            if (cudaMemcpy(sdf_out, sdf.data(), sizeof(float) * nn, cudaMemcpyHostToDevice) != cudaSuccess)
                return set_error(TRIME_ECUDA, "copy of the SDF grid failed");
        } else {
            std::memcpy(sdf_out, sdf.data(), sizeof(float) * nn);
        }
    }
    if (counts) {
        counts[0] = ns;
        counts[1] = (int64_t)M.size() / 2;
        counts[2] = kept;
    }
    return TRIME_OK;
}
