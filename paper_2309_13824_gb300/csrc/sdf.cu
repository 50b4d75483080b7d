// sdf.cu -- the signed distance field of a closed loop of line segments
// given clockwise (TriMe++ Sec. 3.1), sampled on a node grid.
//
// Value at p: the distance to the closest segment (FP64; the smaller segment
// index on ties; closest point p* = a + t (b - a), t the clamped projection),
// negative where (p - p*) . n > 0 with n the segment's inward unit normal
// (right of its direction for a clockwise loop), or, when p* is an end point,
// the sum of the two incident segments' unit normals; rounded to float32.
// Every decision uses fixed FP64 formulas (explicit round-to-nearest
// operations), so the result does not depend on the search order.
//
// Search.  As in the paper, the segments are listed in a grid of cells about
// the mean segment length (each segment in the cells its bounding box
// touches) and searched outwards ring by ring.  A per-node ring search would
// walk many empty cells for nodes far from the boundary, so the search runs
// once per cell instead: the cell's centre c finds an upper bound d_c of its
// distance (the closest segment of the first non-empty ring), then collects
// every segment within d_c + diag of c (diag the cell diagonal).  A node p of
// the cell has distance at most d_c + |p - c|, so its closest segment lies
// within d_c + diag of c: the candidates hold it, and each node evaluates only
// its cell's candidates.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "seg.cuh"
#include "trime.h"

namespace trime {

// segment k's bounding box in cells
__device__ __forceinline__ void seg_cells(const double* xy, int32_t nv, int32_t k, const SegGrid& G, int& i0, int& i1,
                                          int& j0, int& j1) {
    int32_t k1 = k + 1 == nv ? 0 : k + 1;
    double ax = xy[2 * k], ay = xy[2 * k + 1], bx = xy[2 * k1], by = xy[2 * k1 + 1];
    i0 = cell_x(G, fmin(ax, bx));
    i1 = cell_x(G, fmax(ax, bx));
    j0 = cell_y(G, fmin(ay, by));
    j1 = cell_y(G, fmax(ay, by));
}

__global__ void k_seg_count(const double* xy, int32_t nv, SegGrid G, int32_t* cnt) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nv) return;
    int i0, i1, j0, j1;
    seg_cells(xy, nv, k, G, i0, i1, j0, j1);
    for (int j = j0; j <= j1; j++)
        for (int i = i0; i <= i1; i++) atomicAdd(&cnt[j * G.gx + i], 1);
}

__global__ void k_seg_fill(const double* xy, int32_t nv, SegGrid G, const int32_t* start, int32_t* cur,
                           int32_t* list) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nv) return;
    int i0, i1, j0, j1;
    seg_cells(xy, nv, k, G, i0, i1, j0, j1);
    for (int j = j0; j <= j1; j++)
        for (int i = i0; i <= i1; i++) {
            int c = j * G.gx + i;
            list[start[c] + atomicAdd(&cur[c], 1)] = k;
        }
}

// the radius around cell c's centre that holds the closest segment of every
// node of the cell: the closest segment of the first non-empty ring, plus
// the diagonal and a margin for rounding
__device__ double cell_radius(const double* xy, int32_t nv, const SegGrid& G, const int32_t* start,
                              const int32_t* list, int ci, int cj) {
    double cx = G.x0 + (ci + 0.5) * G.cw, cy = G.y0 + (cj + 0.5) * G.ch;
    double best = INFINITY;
    int rmax = max(max(ci, G.gx - 1 - ci), max(cj, G.gy - 1 - cj));
    for (int r = 0; r <= rmax && !(best < INFINITY); r++) {
        for (int j = cj - r; j <= cj + r; j++) {
            if (j < 0 || j >= G.gy) continue;
            int step = (j == cj - r || j == cj + r) ? 1 : 2 * r;
            for (int i = ci - r; i <= ci + r; i += step > 0 ? step : 1) {
                if (i < 0 || i >= G.gx) continue;
                int c = j * G.gx + i;
                for (int q = start[c]; q < start[c + 1]; q++) {
                    double d, t;
                    seg_dist(xy, nv, list[q], cx, cy, d, t);
                    best = fmin(best, d);
                }
            }
        }
    }
    return best + G.diag + 1e-9 * (best + G.diag) + 1e-12;
}

// candidates of cell (ci, cj): segments within R of the centre, each once (a
// segment counts in the lowest-left cell of its box inside the search block)
template <bool kFill>
__device__ int cell_candidates(const double* xy, int32_t nv, const SegGrid& G, const int32_t* start,
                               const int32_t* list, int ci, int cj, double R, int32_t* out) {
    double cx = G.x0 + (ci + 0.5) * G.cw, cy = G.y0 + (cj + 0.5) * G.ch;
    int ri = (int)ceil(R / G.cw) + 1, rj = (int)ceil(R / G.ch) + 1;
    int bi0 = max(0, ci - ri), bi1 = min(G.gx - 1, ci + ri), bj0 = max(0, cj - rj), bj1 = min(G.gy - 1, cj + rj);
    int n = 0;
    for (int j = bj0; j <= bj1; j++)
        for (int i = bi0; i <= bi1; i++) {
            int c = j * G.gx + i;
            for (int q = start[c]; q < start[c + 1]; q++) {
                int k = list[q];
                int i0, i1, j0, j1;
                seg_cells(xy, nv, k, G, i0, i1, j0, j1);
                if (i != max(i0, bi0) || j != max(j0, bj0)) continue;
                double d, t;
                seg_dist(xy, nv, k, cx, cy, d, t);
                if (!(d <= R)) continue;
                if (kFill) out[n] = k;
                n++;
            }
        }
    return n;
}

__global__ void k_cell_count(const double* xy, int32_t nv, SegGrid G, const int32_t* start, const int32_t* list,
                             double* rad, int32_t* ncand) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= G.gx * G.gy) return;
    int ci = c % G.gx, cj = c / G.gx;
    double R = cell_radius(xy, nv, G, start, list, ci, cj);
    rad[c] = R;
    ncand[c] = cell_candidates<false>(xy, nv, G, start, list, ci, cj, R, nullptr);
}

__global__ void k_cell_fill(const double* xy, int32_t nv, SegGrid G, const int32_t* start, const int32_t* list,
                            const double* rad, const int32_t* cstart, int32_t* cand) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= G.gx * G.gy) return;
    cell_candidates<true>(xy, nv, G, start, list, c % G.gx, c / G.gx, rad[c], cand + cstart[c]);
}

__global__ void k_sdf_nodes(const double* xy, int32_t nv, SegGrid G, const int32_t* cstart, const int32_t* cand,
                            double gx0, double gy0, double gdx, double gdy, int32_t nx, int32_t ny, float* out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)nx * ny) return;
    int i = (int)(q % nx), j = (int)(q / nx);
    double x = fadd(gx0, fmul((double)i, gdx)), y = fadd(gy0, fmul((double)j, gdy));
    out[q] = __double2float_rn(seg_sdf_cand(xy, nv, G, cstart, cand, x, y));
}

}  // namespace trime

using namespace trime;

#define SDF_TRY(x)                                                                          \
    do {                                                                                    \
        cudaError_t e_ = (x);                                                               \
        if (e_ != cudaSuccess) {                                                            \
            rc = set_error(TRIME_ECUDA, (std::string(#x) + ": " + cudaGetErrorString(e_)).c_str()); \
            goto done;                                                                      \
        }                                                                                   \
    } while (0)

namespace trime {

void seg_index_free(SegIndex* s) {
    for (void* p : {(void*)s->cnt, (void*)s->start, (void*)s->cur, (void*)s->list, (void*)s->tmp, (void*)s->ncand,
                    (void*)s->cstart, (void*)s->cand, (void*)s->rad})
        if (p) cudaFree(p);
    *s = SegIndex{};
}

int seg_index_build(const double* xy, const double* dxy, int64_t nv, double x0, double y0, double x1, double y1,
                    SegIndex* out, cudaStream_t st) {
    *out = SegIndex{};
    double perim = 0.0;
    for (int64_t k = 0; k < nv; k++) {
        int64_t k1 = k + 1 == nv ? 0 : k + 1;
        perim += std::hypot(xy[2 * k1] - xy[2 * k], xy[2 * k1 + 1] - xy[2 * k + 1]);
    }
    // cells about the mean segment length (Sec. 3.1), at most 2^22 of them
    double lbar = perim / (double)nv, W = x1 - x0, H = y1 - y0;
    double cs = std::max(lbar, std::sqrt(W * H / (double)(1 << 22)));
    SegGrid G;
    G.gx = (int32_t)std::max(1.0, std::ceil(W / cs));
    G.gy = (int32_t)std::max(1.0, std::ceil(H / cs));
    G.x0 = x0;
    G.y0 = y0;
    G.cw = W / G.gx;
    G.ch = H / G.gy;
    G.diag = std::hypot(G.cw, G.ch);
    // the cell lists must fit int32 offsets
    int64_t entries = 0;
    for (int64_t k = 0; k < nv; k++) {
        int64_t k1 = k + 1 == nv ? 0 : k + 1;
        auto cx = [&](double x) { return std::min<int64_t>(G.gx - 1, std::max<int64_t>(0, (int64_t)std::floor((x - x0) / G.cw))); };
        auto cy = [&](double y) { return std::min<int64_t>(G.gy - 1, std::max<int64_t>(0, (int64_t)std::floor((y - y0) / G.ch))); };
        int64_t w = cx(std::max(xy[2 * k], xy[2 * k1])) - cx(std::min(xy[2 * k], xy[2 * k1])) + 1;
        int64_t h = cy(std::max(xy[2 * k + 1], xy[2 * k1 + 1])) - cy(std::min(xy[2 * k + 1], xy[2 * k1 + 1])) + 1;
        entries += w * h;
    }
    if (entries > (int64_t)1 << 30) return set_error(TRIME_EINVAL, "segments cover too many cells");
    int rc = TRIME_OK;
    SegIndex& S = *out;
    S.G = G;
    std::vector<int32_t> hc;
    int32_t ncell = G.gx * G.gy;
    int32_t total = 0, ctotal = 0;
    SDF_TRY(cudaMalloc(&S.cnt, sizeof(int32_t) * ncell));
    SDF_TRY(cudaMalloc(&S.start, sizeof(int32_t) * ((size_t)ncell + 1)));
    SDF_TRY(cudaMalloc(&S.cur, sizeof(int32_t) * ncell));
    SDF_TRY(cudaMalloc(&S.tmp, sizeof(int32_t) * ((size_t)ncell / 4096 + 2)));
    SDF_TRY(cudaMalloc(&S.ncand, sizeof(int32_t) * ncell));
    SDF_TRY(cudaMalloc(&S.cstart, sizeof(int32_t) * ((size_t)ncell + 1)));
    SDF_TRY(cudaMalloc(&S.rad, sizeof(double) * ncell));
    SDF_TRY(cudaMemsetAsync(S.cnt, 0, sizeof(int32_t) * ncell, st));
    SDF_TRY(cudaMemsetAsync(S.cur, 0, sizeof(int32_t) * ncell, st));
    k_seg_count<<<(int)((nv + 255) / 256), 256, 0, st>>>(dxy, (int32_t)nv, G, S.cnt);
    launch_scan(S.cnt, S.start, ncell, S.tmp, st);
    SDF_TRY(cudaMemcpyAsync(&total, S.start + ncell, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SDF_TRY(cudaStreamSynchronize(st));
    SDF_TRY(cudaMalloc(&S.list, sizeof(int32_t) * std::max<int32_t>(total, 1)));
    k_seg_fill<<<(int)((nv + 255) / 256), 256, 0, st>>>(dxy, (int32_t)nv, G, S.start, S.cur, S.list);
    k_cell_count<<<(ncell + 127) / 128, 128, 0, st>>>(dxy, (int32_t)nv, G, S.start, S.list, S.rad, S.ncand);
    hc.resize(ncell);
    SDF_TRY(cudaMemcpyAsync(hc.data(), S.ncand, sizeof(int32_t) * ncell, cudaMemcpyDeviceToHost, st));
    SDF_TRY(cudaStreamSynchronize(st));
    {
        int64_t sum = 0;
        for (int32_t v : hc) sum += v;
        if (sum > (int64_t)1 << 30) {
            rc = set_error(TRIME_EINVAL, "too many candidate segments (shape too large for the cell grid)");
            goto done;
        }
    }
    launch_scan(S.ncand, S.cstart, ncell, S.tmp, st);
    SDF_TRY(cudaMemcpyAsync(&ctotal, S.cstart + ncell, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SDF_TRY(cudaStreamSynchronize(st));
    SDF_TRY(cudaMalloc(&S.cand, sizeof(int32_t) * std::max<int32_t>(ctotal, 1)));
    k_cell_fill<<<(ncell + 127) / 128, 128, 0, st>>>(dxy, (int32_t)nv, G, S.start, S.list, S.rad, S.cstart, S.cand);
    SDF_TRY(cudaGetLastError());
done:
    if (rc) seg_index_free(out);
    return rc;
}

}  // namespace trime

extern "C" int mesh_segment_sdf_grid(const double* xy, int64_t nv, double x0, double y0, double x1, double y1,
                                     int32_t nx, int32_t ny, float* out, void* cuda_stream) {
    if (!xy || !out) return set_error(TRIME_EINVAL, "NULL pointer");
    if (nv < 3 || nv > (int64_t)1 << 26) return set_error(TRIME_EINVAL, "need 3 .. 2^26 vertices");
    if (nx < 2 || ny < 2 || (int64_t)nx * ny > ((int64_t)1 << 31) - 1)
        return set_error(TRIME_EINVAL, "grid must have 2 .. 2^31 nodes, at least 2 per side");
    if (!(x1 > x0) || !(y1 > y0) || !std::isfinite(x0) || !std::isfinite(x1) || !std::isfinite(y0) ||
        !std::isfinite(y1))
        return set_error(TRIME_EINVAL, "bad grid box");
    for (int64_t k = 0; k < nv; k++) {
        int64_t k1 = k + 1 == nv ? 0 : k + 1;
        if (!std::isfinite(xy[2 * k]) || !std::isfinite(xy[2 * k + 1]))
            return set_error(TRIME_EINVAL, "vertices must be finite");
        double L = std::hypot(xy[2 * k1] - xy[2 * k], xy[2 * k1 + 1] - xy[2 * k + 1]);
        if (!(L > 0.0)) return set_error(TRIME_EINVAL, "zero-length segment");
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc = TRIME_OK;
    size_t nn = (size_t)nx * (size_t)ny;
    double* dxy = nullptr;
    float* dout = nullptr;
    SegIndex S;
    cudaPointerAttributes at;
    bool dev_out = cudaPointerGetAttributes(&at, out) == cudaSuccess &&
                   (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    SDF_TRY(cudaMalloc(&dxy, sizeof(double) * 2 * (size_t)nv));
    SDF_TRY(cudaMemcpyAsync(dxy, xy, sizeof(double) * 2 * (size_t)nv, cudaMemcpyHostToDevice, st));
    if ((rc = seg_index_build(xy, dxy, nv, x0, y0, x1, y1, &S, st))) goto done;
    if (dev_out) dout = out;
    else SDF_TRY(cudaMalloc(&dout, sizeof(float) * nn));
    k_sdf_nodes<<<(int)((nn + 255) / 256), 256, 0, st>>>(dxy, (int32_t)nv, S.G, S.cstart, S.cand, x0, y0,
                                                         (x1 - x0) / (double)(nx - 1), (y1 - y0) / (double)(ny - 1),
                                                         nx, ny, dout);
    SDF_TRY(cudaGetLastError());
    if (!dev_out) SDF_TRY(cudaMemcpyAsync(out, dout, sizeof(float) * nn, cudaMemcpyDeviceToHost, st));
    SDF_TRY(cudaStreamSynchronize(st));
done:
    cudaStreamSynchronize(st);
    seg_index_free(&S);
    if (dxy) cudaFree(dxy);
    if (dout && !dev_out) cudaFree(dout);
    return rc;
}
