// quality.cu -- the mesh-quality report of one mesh's last rebuild (Sec. 3.6
// Eqs. 11-12 quality measures and the statistics the paper tabulates at
// termination, Sec. 5: median, mean, maximum and standard deviation of the
// triangles' aspect ratio alpha = R_circ / (2 R_in) and edge ratio
// beta = l_max / l_min, the share of triangles with alpha < 1.2 and < 2),
// plus the minimum angle, a histogram of alpha, and the deviation of the
// valid edges' lengths from the sizing field, |l / (fac_mu mu(m)) - 1|
// (Eq. 3), by mean and 95th percentile.
//
// Every value is computed in FP64 at the positions the rebuild triangulated.
// One thread per owner slot writes the values of the valid triangles and the
// valid edges it owns (smallest id) at offsets from a count and a scan; the
// sums are per-block partials added in a fixed order (alpha and beta shifted
// by 1, which they never go below, so the variance does not cancel); medians
// and the percentile are exact order statistics found by a most-significant-
// byte-first radix select over the bit patterns of the non-negative doubles
// (one 256-bin histogram per byte).
#include <cstring>
#include <string>

#include <algorithm>
#include <cmath>

#include "kernels.cuh"
#include "trime.h"

namespace trime {

constexpr int kQBins = 10;
// alpha histogram edges: bin k holds alpha in [e_k, e_{k+1}), e_0 = 1 (alpha
// >= 1; rounding below 1 counts in bin 0), the last bin is open
__constant__ double kQEdge[kQBins] = {1.0, 1.05, 1.1, 1.2, 1.3, 1.5, 2.0, 3.0, 5.0, 10.0};

struct QPartial {
    double sa, sa2, sb, sb2, amax, bmax, angmin, sdev;
    long long n_lt12, n_lt2, hist[kQBins];
};

template <typename T>
__global__ void k_q_count(const __grid_constant__ IterArgs<T> a, int32_t s0, int32_t ns, int32_t* tcnt,
                          int32_t* ecnt) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ns) return;
    int s = s0 + r;
    int ne = a.ring_n[s];
    uint64_t vm = a.vmask[s];
    int idi = a.srt.id[s];
    int ct = 0, ce = 0;
    for (int t = 0; t < ne; t++) {
        int j = a.ring[(size_t)s * kRingCap + t];
        int tp = t == 0 ? ne - 1 : t - 1;
        if (j < 0) continue;
        if (((vm >> t) & 1ull) || ((vm >> tp) & 1ull))
            if (idi < a.srt.id[j]) ce++;  // a valid edge, counted by its smaller id
        if (!((vm >> t) & 1ull)) continue;
        int k = a.ring[(size_t)s * kRingCap + (t + 1 == ne ? 0 : t + 1)];
        if (idi < a.srt.id[j] && idi < a.srt.id[k]) ct++;
    }
    tcnt[r] = ct;
    ecnt[r] = ce;
}

template <typename T>
__global__ void k_q_values(const __grid_constant__ IterArgs<T> a, int32_t s0, int32_t ns, const int32_t* toff,
                           const int32_t* eoff, double fac_mu, double* alpha, double* beta, double* ang,
                           double* dev) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ns) return;
    int s = s0 + r;
    const MeshView& V = a.Vs ? a.Vs[__ldg(a.cmesh + (s >> kChunkShift))] : a.V;  // the slot's mesh
    int ne = a.ring_n[s];
    uint64_t vm = a.vmask[s];
    int idi = a.srt.id[s];
    const double xi = (double)a.srt.x[s], yi = (double)a.srt.y[s];
    int ot = toff[r], oe = eoff[r];
    for (int t = 0; t < ne; t++) {
        int j = a.ring[(size_t)s * kRingCap + t];
        int tp = t == 0 ? ne - 1 : t - 1;
        if (j < 0) continue;
        const double xj = (double)a.srt.x[j], yj = (double)a.srt.y[j];
        if ((((vm >> t) & 1ull) || ((vm >> tp) & 1ull)) && idi < a.srt.id[j]) {
            double dx = xj - xi, dy = yj - yi;
            double l = sqrt(dx * dx + dy * dy);
            double mu = bilin<double>(V.siz, (xi + xj) * 0.5, (yi + yj) * 0.5);
            dev[oe++] = fabs(l / (fac_mu * mu) - 1.0);
        }
        if (!((vm >> t) & 1ull)) continue;
        int k = a.ring[(size_t)s * kRingCap + (t + 1 == ne ? 0 : t + 1)];
        if (!(idi < a.srt.id[j] && idi < a.srt.id[k])) continue;
        const double xk = (double)a.srt.x[k], yk = (double)a.srt.y[k];
        // side lengths opposite i, j, k
        double la = sqrt((xj - xk) * (xj - xk) + (yj - yk) * (yj - yk));
        double lb = sqrt((xk - xi) * (xk - xi) + (yk - yi) * (yk - yi));
        double lc = sqrt((xi - xj) * (xi - xj) + (yi - yj) * (yi - yj));
        double o = (xj - xi) * (yk - yi) - (yj - yi) * (xk - xi);
        double A = 0.5 * fabs(o);
        alpha[ot] = (la * lb * lc * (la + lb + lc)) / (16.0 * A * A);  // R / (2 r)
        double lmax = fmax(la, fmax(lb, lc)), lmin = fmin(la, fmin(lb, lc));
        beta[ot] = lmax / lmin;
        // the smallest angle lies opposite the shortest side (law of cosines)
        double p, q;
        if (lmin == la) p = lb, q = lc;
        else if (lmin == lb) p = la, q = lc;
        else p = la, q = lb;
        double cs = (p * p + q * q - lmin * lmin) / (2.0 * p * q);
        cs = fmin(fmax(cs, -1.0), 1.0);
        ang[ot] = acos(cs) * (180.0 / 3.141592653589793);
        ot++;
    }
}

constexpr int kQThreads = 256;

__global__ void __launch_bounds__(kQThreads) k_q_sums(const double* alpha, const double* beta, const double* ang,
                                                      int32_t nt, const double* dev, int32_t nedge, QPartial* part) {
    QPartial p{};
    p.angmin = 180.0;
    int stride = gridDim.x * kQThreads;
    for (int i = blockIdx.x * kQThreads + threadIdx.x; i < nt; i += stride) {
        double x = alpha[i] - 1.0, y = beta[i] - 1.0;
        p.sa += x;
        p.sa2 += x * x;
        p.sb += y;
        p.sb2 += y * y;
        p.amax = fmax(p.amax, alpha[i]);
        p.bmax = fmax(p.bmax, beta[i]);
        p.angmin = fmin(p.angmin, ang[i]);
        p.n_lt12 += alpha[i] < 1.2;
        p.n_lt2 += alpha[i] < 2.0;
        int b = 0;
#pragma unroll
        for (int k = 1; k < kQBins; k++) b += alpha[i] >= kQEdge[k];
        p.hist[b]++;
    }
    for (int i = blockIdx.x * kQThreads + threadIdx.x; i < nedge; i += stride) p.sdev += dev[i];
    // block reduction in a fixed order through shared memory
    __shared__ QPartial sh[kQThreads];
    sh[threadIdx.x] = p;
    __syncthreads();
    for (int w = kQThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            QPartial& u = sh[threadIdx.x];
            const QPartial& v = sh[threadIdx.x + w];
            u.sa += v.sa;
            u.sa2 += v.sa2;
            u.sb += v.sb;
            u.sb2 += v.sb2;
            u.amax = fmax(u.amax, v.amax);
            u.bmax = fmax(u.bmax, v.bmax);
            u.angmin = fmin(u.angmin, v.angmin);
            u.sdev += v.sdev;
            u.n_lt12 += v.n_lt12;
            u.n_lt2 += v.n_lt2;
            for (int k = 0; k < kQBins; k++) u.hist[k] += v.hist[k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// one 256-bin histogram of byte `shift` of the bit patterns of v[0..n) whose
// bits above that byte equal `prefix`
__global__ void __launch_bounds__(kQThreads) k_q_hist(const double* v, int32_t n, unsigned long long prefix,
                                                      unsigned long long mask, int shift, unsigned int* hist) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    for (int i = blockIdx.x * kQThreads + threadIdx.x; i < n; i += gridDim.x * kQThreads) {
        unsigned long long b = (unsigned long long)__double_as_longlong(v[i]);
        if ((b & mask) == prefix) atomicAdd(&h[(b >> shift) & 0xFFull], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

constexpr int kQParts = 152;

#define Q_TRY(x)                                              \
    do {                                                      \
        cudaError_t e_ = (x);                                 \
        if (e_ != cudaSuccess) {                              \
            err = cudaGetErrorString(e_);                     \
            return -1;                                        \
        }                                                     \
    } while (0)

// k-th smallest of v[0..n) (0 <= k < n, every value >= 0) by radix select
static int q_select(const double* v, int32_t n, int64_t k, const QBufs& b, cudaStream_t st, double& out,
                    std::string& err) {
    unsigned long long prefix = 0, mask = 0;
    int g = (n + kQThreads - 1) / kQThreads;
    if (g > 4 * kQParts) g = 4 * kQParts;
    for (int shift = 56; shift >= 0; shift -= 8) {
        Q_TRY(cudaMemsetAsync(b.hist, 0, 256 * sizeof(unsigned int), st));
        k_q_hist<<<g, kQThreads, 0, st>>>(v, n, prefix, mask, shift, b.hist);
        Q_TRY(cudaMemcpyAsync(b.hhist, b.hist, 256 * sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
        Q_TRY(cudaStreamSynchronize(st));
        int bin = 0;
        for (; bin < 256; bin++) {
            if (k < (int64_t)b.hhist[bin]) break;
            k -= b.hhist[bin];
        }
        if (bin == 256) {
            err = "order statistic out of range";
            return -2;
        }
        prefix |= (unsigned long long)bin << shift;
        mask |= 0xFFull << shift;
    }
    std::memcpy(&out, &prefix, sizeof out);
    return 0;
}

template <typename T>
int quality_report(const IterArgs<T>& a, int32_t s0, int32_t ns, double fac_mu, const QBufs& b, int64_t cap_t,
                   int64_t cap_e, cudaStream_t st, mesh_quality_stats* q, std::string& err) {
    std::memset(q, 0, sizeof *q);
    q->fac_mu = fac_mu;
    if (ns <= 0) return 0;
    int g = (ns + kQThreads - 1) / kQThreads;
    k_q_count<T><<<g, kQThreads, 0, st>>>(a, s0, ns, b.tcnt, b.ecnt);
    launch_scan(b.tcnt, b.toff, ns, b.scan_tmp, st);
    launch_scan(b.ecnt, b.eoff, ns, b.scan_tmp, st);
    int32_t tot[2] = {0, 0};
    Q_TRY(cudaMemcpyAsync(&tot[0], b.toff + ns, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    Q_TRY(cudaMemcpyAsync(&tot[1], b.eoff + ns, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    Q_TRY(cudaStreamSynchronize(st));
    const int32_t nt = tot[0], nedge = tot[1];
    if (nt > cap_t || nedge > cap_e) {
        err = "more valid triangles or edges than the report's buffers hold";
        return -2;
    }
    q->n_tri = nt;
    q->n_edges = nedge;
    if (nt == 0 && nedge == 0) return 0;
    k_q_values<T><<<g, kQThreads, 0, st>>>(a, s0, ns, b.toff, b.eoff, fac_mu, b.alpha, b.beta, b.ang, b.dev);
    k_q_sums<<<kQParts, kQThreads, 0, st>>>(b.alpha, b.beta, b.ang, nt, b.dev, nedge, b.part);
    Q_TRY(cudaGetLastError());
    QPartial hp[kQParts];
    Q_TRY(cudaMemcpyAsync(hp, b.part, sizeof hp, cudaMemcpyDeviceToHost, st));
    Q_TRY(cudaStreamSynchronize(st));
    // the partials of the fixed block order, added in that order
    QPartial t = hp[0];
    for (int k = 1; k < kQParts; k++) {
        t.sa += hp[k].sa;
        t.sa2 += hp[k].sa2;
        t.sb += hp[k].sb;
        t.sb2 += hp[k].sb2;
        t.amax = std::max(t.amax, hp[k].amax);
        t.bmax = std::max(t.bmax, hp[k].bmax);
        t.angmin = std::min(t.angmin, hp[k].angmin);
        t.sdev += hp[k].sdev;
        t.n_lt12 += hp[k].n_lt12;
        t.n_lt2 += hp[k].n_lt2;
        for (int j = 0; j < kQBins; j++) t.hist[j] += hp[k].hist[j];
    }
    if (nt > 0) {
        double n = (double)nt, ma = t.sa / n, mb = t.sb / n;
        q->mean_alpha = 1.0 + ma;
        q->mean_beta = 1.0 + mb;
        q->std_alpha = std::sqrt(std::max(t.sa2 / n - ma * ma, 0.0));
        q->std_beta = std::sqrt(std::max(t.sb2 / n - mb * mb, 0.0));
        q->max_alpha = t.amax;
        q->max_beta = t.bmax;
        q->min_angle_deg = t.angmin;
        q->frac_alpha_lt_1_2 = (double)t.n_lt12 / n;
        q->frac_alpha_lt_2 = (double)t.n_lt2 / n;
        for (int j = 0; j < kQBins; j++) q->alpha_hist[j] = t.hist[j];
        int rc = q_select(b.alpha, nt, (nt - 1) / 2, b, st, q->median_alpha, err);
        if (!rc) rc = q_select(b.beta, nt, (nt - 1) / 2, b, st, q->median_beta, err);
        if (rc) return rc;
    }
    if (nedge > 0) {
        q->mean_size_dev = t.sdev / (double)nedge;
        // 95th percentile by the nearest rank: the value of rank ceil(0.95 n)
        int64_t r = (int64_t)std::ceil(0.95 * (double)nedge) - 1;
        int rc = q_select(b.dev, nedge, r < 0 ? 0 : r, b, st, q->p95_size_dev, err);
        if (rc) return rc;
    }
    return 0;
}

template int quality_report<double>(const IterArgs<double>&, int32_t, int32_t, double, const QBufs&, int64_t, int64_t,
                                    cudaStream_t, mesh_quality_stats*, std::string&);
template int quality_report<float>(const IterArgs<float>&, int32_t, int32_t, double, const QBufs&, int64_t, int64_t,
                                   cudaStream_t, mesh_quality_stats*, std::string&);

}  // namespace trime
