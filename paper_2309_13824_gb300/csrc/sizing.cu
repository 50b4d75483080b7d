// sizing.cu -- the element sizing field of TriMe++ Eq. 7 (Sec. 3.3) on a node
// grid: mu(x) = min over the boundary samples s of K |s - x| + lfs(s).
//
// The samples sit in a bucket grid; each node searches it outwards ring by
// ring and stops once no unvisited sample can do better: a sample outside the
// visited block is at least the block's distance D away, so its value is at
// least K D + min(lfs).  Values use one fixed FP64 formula (explicit
// round-to-nearest operations), so the result does not depend on the search
// order; rounded to float32.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "trime.h"

namespace trime {

struct SampleGrid {
    double x0, y0, bw, bh;
    int32_t gx, gy;
};

__device__ __forceinline__ int sbucket(double v, double v0, double b, int g) {
    double f = floor((v - v0) / b);
    return f < 0.0 ? 0 : (f > (double)(g - 1) ? g - 1 : (int)f);
}

__global__ void k_smp_count(const double* sxy, int32_t ns, SampleGrid G, int32_t* cnt) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ns) return;
    int i = sbucket(sxy[2 * k], G.x0, G.bw, G.gx), j = sbucket(sxy[2 * k + 1], G.y0, G.bh, G.gy);
    atomicAdd(&cnt[j * G.gx + i], 1);
}

__global__ void k_smp_fill(const double* sxy, int32_t ns, SampleGrid G, const int32_t* start, int32_t* cur,
                           int32_t* list) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ns) return;
    int i = sbucket(sxy[2 * k], G.x0, G.bw, G.gx), j = sbucket(sxy[2 * k + 1], G.y0, G.bh, G.gy);
    int c = j * G.gx + i;
    list[start[c] + atomicAdd(&cur[c], 1)] = k;
}

__global__ void k_sizing_nodes(const double* sxy, const double* lfs, SampleGrid G, const int32_t* start,
                               const int32_t* list, double K, double lfs_min, double gx0, double gy0, double gdx,
                               double gdy, int32_t nx, int32_t ny, float* out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)nx * ny) return;
    int i = (int)(q % nx), j = (int)(q / nx);
    double x = fadd(gx0, fmul((double)i, gdx)), y = fadd(gy0, fmul((double)j, gdy));
    int ci = sbucket(x, G.x0, G.bw, G.gx), cj = sbucket(y, G.y0, G.bh, G.gy);
    double best = INFINITY;
    for (int r = 0;; r++) {
        for (int jj = cj - r; jj <= cj + r; jj++) {
            if (jj < 0 || jj >= G.gy) continue;
            int step = (jj == cj - r || jj == cj + r) ? 1 : 2 * r;
            for (int ii = ci - r; ii <= ci + r; ii += step) {
                if (ii < 0 || ii >= G.gx) continue;
                int c = jj * G.gx + ii;
                for (int u = start[c]; u < start[c + 1]; u++) {
                    int k = list[u];
                    double dx = fsub(x, sxy[2 * k]), dy = fsub(y, sxy[2 * k + 1]);
                    double v = fadd(fmul(K, __dsqrt_rn(fadd(fmul(dx, dx), fmul(dy, dy)))), lfs[k]);
                    best = fmin(best, v);
                }
            }
        }
        // distance to the region outside the visited block (sides at the grid edge are closed)
        double D = INFINITY;
        if (ci - r > 0) D = fmin(D, x - (G.x0 + (ci - r) * G.bw));
        if (ci + r < G.gx - 1) D = fmin(D, (G.x0 + (ci + r + 1) * G.bw) - x);
        if (cj - r > 0) D = fmin(D, y - (G.y0 + (cj - r) * G.bh));
        if (cj + r < G.gy - 1) D = fmin(D, (G.y0 + (cj + r + 1) * G.bh) - y);
        if (!(D < INFINITY)) break;  // the whole grid is visited
        if (best <= K * D * (1.0 - 1e-9) + lfs_min) break;
    }
    out[q] = __double2float_rn(best);
}

}  // namespace trime

using namespace trime;

#define SZ_TRY(x)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (x);                                                                       \
        if (e_ != cudaSuccess) {                                                                    \
            rc = set_error(TRIME_ECUDA, (std::string(#x) + ": " + cudaGetErrorString(e_)).c_str()); \
            goto done;                                                                              \
        }                                                                                           \
    } while (0)

extern "C" int mesh_sizing_field(const double* sxy, const double* lfs, int64_t ns, double K, double x0, double y0,
                                 double x1, double y1, int32_t nx, int32_t ny, float* out, void* cuda_stream) {
    if (!sxy || !lfs || !out) return set_error(TRIME_EINVAL, "NULL pointer");
    if (ns < 1 || ns > (int64_t)1 << 28) return set_error(TRIME_EINVAL, "need 1 .. 2^28 samples");
    if (!(K >= 0.0) || !std::isfinite(K)) return set_error(TRIME_EINVAL, "K must be finite and >= 0");
    if (nx < 2 || ny < 2 || (int64_t)nx * ny > ((int64_t)1 << 31) - 1)
        return set_error(TRIME_EINVAL, "grid must have 2 .. 2^31 nodes, at least 2 per side");
    if (!(x1 > x0) || !(y1 > y0) || !std::isfinite(x0) || !std::isfinite(x1) || !std::isfinite(y0) ||
        !std::isfinite(y1))
        return set_error(TRIME_EINVAL, "bad grid box");
    double lfs_min = INFINITY;
    for (int64_t k = 0; k < ns; k++) {
        if (!std::isfinite(sxy[2 * k]) || !std::isfinite(sxy[2 * k + 1]) || !(lfs[k] >= 0.0) || !std::isfinite(lfs[k]))
            return set_error(TRIME_EINVAL, "samples and lfs must be finite, lfs >= 0");
        lfs_min = std::min(lfs_min, lfs[k]);
    }
    // about one sample per bucket, at most 2^22 buckets
    double W = x1 - x0, H = y1 - y0;
    double bs = std::max(std::sqrt(W * H / (double)ns), std::sqrt(W * H / (double)(1 << 22)));
    SampleGrid G;
    G.gx = (int32_t)std::max(1.0, std::ceil(W / bs));
    G.gy = (int32_t)std::max(1.0, std::ceil(H / bs));
    G.x0 = x0;
    G.y0 = y0;
    G.bw = W / G.gx;
    G.bh = H / G.gy;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc = TRIME_OK;
    int32_t nb = G.gx * G.gy;
    size_t nn = (size_t)nx * (size_t)ny;
    double *dxy = nullptr, *dlfs = nullptr;
    int32_t *cnt = nullptr, *start = nullptr, *cur = nullptr, *list = nullptr, *tmp = nullptr;
    float* dout = nullptr;
    cudaPointerAttributes at;
    bool dev_out = cudaPointerGetAttributes(&at, out) == cudaSuccess &&
                   (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    SZ_TRY(cudaMalloc(&dxy, sizeof(double) * 2 * (size_t)ns));
    SZ_TRY(cudaMalloc(&dlfs, sizeof(double) * (size_t)ns));
    SZ_TRY(cudaMalloc(&cnt, sizeof(int32_t) * nb));
    SZ_TRY(cudaMalloc(&start, sizeof(int32_t) * ((size_t)nb + 1)));
    SZ_TRY(cudaMalloc(&cur, sizeof(int32_t) * nb));
    SZ_TRY(cudaMalloc(&tmp, sizeof(int32_t) * ((size_t)nb / 4096 + 2)));
    SZ_TRY(cudaMalloc(&list, sizeof(int32_t) * (size_t)ns));
    SZ_TRY(cudaMemcpyAsync(dxy, sxy, sizeof(double) * 2 * (size_t)ns, cudaMemcpyHostToDevice, st));
    SZ_TRY(cudaMemcpyAsync(dlfs, lfs, sizeof(double) * (size_t)ns, cudaMemcpyHostToDevice, st));
    SZ_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * nb, st));
    SZ_TRY(cudaMemsetAsync(cur, 0, sizeof(int32_t) * nb, st));
    k_smp_count<<<(int)((ns + 255) / 256), 256, 0, st>>>(dxy, (int32_t)ns, G, cnt);
    launch_scan(cnt, start, nb, tmp, st);
    k_smp_fill<<<(int)((ns + 255) / 256), 256, 0, st>>>(dxy, (int32_t)ns, G, start, cur, list);
    if (dev_out) dout = out;
    else SZ_TRY(cudaMalloc(&dout, sizeof(float) * nn));
    k_sizing_nodes<<<(int)((nn + 255) / 256), 256, 0, st>>>(dxy, dlfs, G, start, list, K, lfs_min, x0, y0,
                                                            (x1 - x0) / (double)(nx - 1),
                                                            (y1 - y0) / (double)(ny - 1), nx, ny, dout);
    SZ_TRY(cudaGetLastError());
    if (!dev_out) SZ_TRY(cudaMemcpyAsync(out, dout, sizeof(float) * nn, cudaMemcpyDeviceToHost, st));
    SZ_TRY(cudaStreamSynchronize(st));
done:
    for (void* p : {(void*)dxy, (void*)dlfs, (void*)cnt, (void*)start, (void*)cur, (void*)list, (void*)tmp})
        if (p) cudaFree(p);
    if (dout && !dev_out) cudaFree(dout);
    return rc;
}
