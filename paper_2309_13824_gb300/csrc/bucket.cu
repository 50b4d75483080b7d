// bucket.cu -- a1: counting sort of the points into the neighbour-bucket grid
// (the paper's Voro++ container of N/N_opt blocks, Sec. 3.2 and Listing 1),
// plus the per-slot precomputation the later kernels read: the geometry cell
// by the fixed formula and the exact-duplicate (SoS) flag.
//
// count: one atomic per point gives its bucket and a provisional rank; scan:
// exclusive prefix over the bucket counts (three passes); place: each point
// writes its index at bucket_start[key] + provisional rank, so a bucket's
// members are listed together (in the atomics' order); scatter: each point
// moves its whole state to bucket_start[key] + the number of the bucket's
// members with a smaller index.  The sort is therefore stable and every
// iteration is bit-reproducible (the provisional ranks come from atomics and
// change from run to run).  All passes are HBM-streaming; the stable rank
// reads the point's bucket list (a few entries) once more.
#include <mutex>

#include "kernels.cuh"
#include "trime.h"

namespace trime {

// One thread per point.  In a batch, a mesh whose iterations have ended, or
// that keeps its last triangulation this iteration, keeps its sorted order:
// its slots all count into its pad bucket, so the offsets of the meshes after
// it stay put; the padding slots of a live mesh count there too.
template <typename T, bool B>
__global__ void __launch_bounds__(kThreads) k_count(const __grid_constant__ IterArgs<T> a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const MeshView& V = mesh_of<B>(a, i);
    bool term = skip_rebuild(V.ctrl, a.force);
    if constexpr (B) {
        int loc = i - V.soff;
        if (term) {
            if (loc == 0) a.bcount[V.boff + V.nb] = V.n + V.npad;
            return;
        }
        if (loc >= V.n) {
            if (loc == V.n) a.bcount[V.boff + V.nb] = V.npad;
            return;
        }
    } else {
        if (term) return;
    }
    int bx, by;
    bucket_of(V.P, a.cur.x[i], a.cur.y[i], bx, by);
    int k = V.boff + by * V.P.nbx + bx;
    a.key[i] = k;
    a.rank[i] = atomicAdd(&a.bcount[k], 1);
}

// the bucket's members listed together (provisional order)
template <typename T, bool B>
__global__ void __launch_bounds__(kThreads) k_place(const __grid_constant__ IterArgs<T> a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const MeshView& V = mesh_of<B>(a, i);
    if (skip_rebuild(V.ctrl, a.force)) return;
    if (B && i - V.soff >= V.n) return;
    a.sidx[a.bstart[a.key[i]] + a.rank[i]] = i;
}

// ------------------------------------------------------------------ scan
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;  // per thread
constexpr int kScanTile = kScanBlock * kScanItems;

__device__ __forceinline__ int block_excl_scan(int v, int* sh, int& total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < (blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    int base = w > 0 ? sh[w - 1] : 0;
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + x - v;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_reduce(const int32_t* in, int32_t n, int32_t* tile_sums) {
    __shared__ int sh[32];
    int base = blockIdx.x * kScanTile;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        int i = base + k * kScanBlock + threadIdx.x;
        if (i < n) s += in[i];
    }
    int total;
    block_excl_scan(s, sh, total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_tiles(int32_t* tile_sums, int32_t ntiles) {
    __shared__ int sh[32];
    int carry = 0;
    for (int b = 0; b < ntiles; b += kScanBlock) {
        int i = b + threadIdx.x;
        int v = i < ntiles ? tile_sums[i] : 0;
        int total;
        int e = block_excl_scan(v, sh, total);
        if (i < ntiles) tile_sums[i] = carry + e;
        carry += total;
    }
}

// out[i] = sum in[0..i), out[n] = total; items of a tile are blocked per thread
__global__ void __launch_bounds__(kScanBlock) k_scan_down(const int32_t* in, int32_t* out, int32_t n,
                                                           const int32_t* tile_off) {
    __shared__ int sh[32];
    int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        int i = base + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    int total;
    int e = block_excl_scan(s, sh, total) + tile_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        int i = base + k;
        if (i < n) out[i] = e;
        if (i == n - 1) out[n] = e + v[k];
        e += v[k];
    }
}

void launch_scan(const int32_t* in, int32_t* out, int32_t n, int32_t* tmp, cudaStream_t st) {
    int ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles < 1) ntiles = 1;
    k_scan_reduce<<<ntiles, kScanBlock, 0, st>>>(in, n, tmp);
    k_scan_tiles<<<1, kScanBlock, 0, st>>>(tmp, ntiles);
    k_scan_down<<<ntiles, kScanBlock, 0, st>>>(in, out, n, tmp);
}

// ------------------------------------------------------------------ scatter
template <typename T, bool B>
__global__ void __launch_bounds__(kThreads) k_scatter(const __grid_constant__ IterArgs<T> a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const MeshView& V = mesh_of<B>(a, i);
    if (skip_rebuild(V.ctrl, a.force)) return;
    if (B && i - V.soff >= V.n) return;
    int k = a.key[i];
    // stable rank: the bucket's members with a smaller index come first
    const int lo = a.bstart[k], hi = a.bstart[k + 1];
    int d = lo;
    for (int q = lo; q < hi; q++) d += a.sidx[q] < i;
    a.perm[i] = d;
    {
        // the point's cell edges at the last rebuild in ring order (old
        // slots, or bounding-plane labels): the clipping pass starts from them
        const int nr = a.ring_n[i];
        const int32_t* row = a.ring + (size_t)i * kRingCap;
        int32_t* wr = a.warm + (size_t)d * kWarm;
        int c = 0;
        for (; c < nr && c < kWarm; c++) wr[c] = row[c];
        for (; c < kWarm; c++) wr[c] = kNoLabel;
    }
    T x = a.cur.x[i], y = a.cur.y[i];
    a.srt.x[d] = x;
    a.srt.y[d] = y;
    a.srt.id[d] = a.cur.id[i];
    a.srt.cls[d] = a.cur.cls[i];
    a.srt.dprev[d] = a.cur.dprev[i];
    a.skey[d] = k;
    // geometry cell by the fixed formula floor((x - x0) / dx); the cheaper
    // product with 1/dx decides unless it lands within 1e-9 of a cell edge
    const DevGrid& sg = V.sdf;
    double xd = (double)x, yd = (double)y;
    double tx = (xd - sg.x0) * (1.0 / sg.dx), ty = (yd - sg.y0) * (1.0 / sg.dy);
    double ftx = tx - floor(tx), fty = ty - floor(ty);
    int gi, gj;
    int ncx = sg.nx - 1, ncy = sg.ny - 1;
    if (ftx > 1e-9 && ftx < 1.0 - 1e-9 && fty > 1e-9 && fty < 1.0 - 1e-9 && tx >= 0.0 && ty >= 0.0 &&
        tx < (double)ncx && ty < (double)ncy) {
        gi = (int)tx;
        gj = (int)ty;
    } else {
        point_cell_fixed(sg, xd, yd, gi, gj);
    }
    a.cell[d] = gj * ncx + gi;
    // per-slot float data read by the cell kernels (computed once per point)
    float xh = (float)x, yh = (float)y;
    double rx = xd - (double)xh, ry = yd - (double)yh;  // exact
    float xl = (float)rx, yl = (float)ry;
    a.pf[d] = make_float4(xh, xl, yh, yl);
    // the remainders below xlo, ylo have at most 5 significant bits: exact
    a.pf3[d] = make_float2((float)(rx - (double)xl), (float)(ry - (double)yl));
    a.pS[d] = (float)(V.P.fac_voro_bound * V.gh[gj * ncx + gi]);
}

// SoS duplicate rule: of several points at exactly the same position the one
// with the largest id owns the cell; the others are flagged (empty cells).
// The 32 slots of a warp belong to one mesh.
template <typename T, bool B>
__global__ void __launch_bounds__(kThreads) k_dups(const __grid_constant__ IterArgs<T> a) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    int sv = s < a.n ? s : a.n - 1;
    const MeshView& V = mesh_of<B>(a, sv);
    if (skip_rebuild(V.ctrl, a.force)) return;
    unsigned dup = 0;
    if (s < a.n && (!B || s - V.soff < V.n)) {
        int k = a.skey[s];
        T x = a.srt.x[s], y = a.srt.y[s];
        int id = a.srt.id[s];
        int e = a.bstart[k + 1];
        for (int q = a.bstart[k]; q < e; q++)
            if (q != s && a.srt.x[q] == x && a.srt.y[q] == y && a.srt.id[q] > id) dup = 1;
        a.dom[s] = (uint8_t)dup;
        // previous neighbours to this rebuild's slots (bounding-plane labels
        // stay); a slot outside the mesh's own slots becomes an empty entry
        int4* w4 = reinterpret_cast<int4*>(a.warm + (size_t)s * kWarm);
        const int lo = V.soff, hi = V.soff + V.n;
        auto map = [&](int l) { return l < 0 ? l : (l >= lo && l < hi ? a.perm[l] : kNoLabel); };
#pragma unroll
        for (int h = 0; h < kWarm / 4; h++) {
            int4 w = w4[h];
            w.x = map(w.x);
            w.y = map(w.y);
            w.z = map(w.z);
            w.w = map(w.w);
            w4[h] = w;
        }
    }
    unsigned m = __ballot_sync(0xffffffffu, dup);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&V.ctrl->cnt.dup_points, (unsigned long long)__popc(m));
}

template <typename T>
void launch_bucket(const IterArgs<T>& a, cudaStream_t st) {
    int g = (a.n + kThreads - 1) / kThreads;
    if (g < 1) g = 1;
    cudaMemsetAsync(a.bcount, 0, sizeof(int32_t) * (size_t)a.nbtot, st);
    if (a.Vs) {
        k_count<T, true><<<g, kThreads, 0, st>>>(a);
        launch_scan(a.bcount, a.bstart, a.nbtot, a.scan_tmp, st);
        k_place<T, true><<<g, kThreads, 0, st>>>(a);
        k_scatter<T, true><<<g, kThreads, 0, st>>>(a);
        k_dups<T, true><<<g, kThreads, 0, st>>>(a);
    } else {
        k_count<T, false><<<g, kThreads, 0, st>>>(a);
        launch_scan(a.bcount, a.bstart, a.nbtot, a.scan_tmp, st);
        k_place<T, false><<<g, kThreads, 0, st>>>(a);
        k_scatter<T, false><<<g, kThreads, 0, st>>>(a);
        k_dups<T, false><<<g, kThreads, 0, st>>>(a);
    }
}

template void launch_bucket<double>(const IterArgs<double>&, cudaStream_t);
template void launch_bucket<float>(const IterArgs<float>&, cudaStream_t);

// ------------------------------------------------------------------ permutations
// cur slots [s0, s0 + ns) hold one mesh whose ids start at s0
template <typename T>
__global__ void k_unpermute(const __grid_constant__ IterArgs<T> a, int32_t s0, int32_t ns, T* out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    s += s0;
    size_t id = (size_t)(a.cur.id[s] - s0);
    out[2 * id] = a.cur.x[s];
    out[2 * id + 1] = a.cur.y[s];
}

template <typename T>
void launch_unpermute(const IterArgs<T>& a, int32_t s0, int32_t ns, T* out, cudaStream_t st) {
    int g = (ns + kThreads - 1) / kThreads;
    if (g > 0) k_unpermute<T><<<g, kThreads, 0, st>>>(a, s0, ns, out);
}
template void launch_unpermute<double>(const IterArgs<double>&, int32_t, int32_t, double*, cudaStream_t);
template void launch_unpermute<float>(const IterArgs<float>&, int32_t, int32_t, float*, cudaStream_t);

template <typename T>
__global__ void k_set_state(const __grid_constant__ IterArgs<T> a, int32_t s0, int32_t ns, const T* xy,
                            const uint8_t* cls, const double* dprev) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    s += s0;
    size_t id = (size_t)(a.cur.id[s] - s0);
    if (xy) {
        a.cur.x[s] = xy[2 * id];
        a.cur.y[s] = xy[2 * id + 1];
    }
    if (cls) a.cur.cls[s] = cls[id];
    if (dprev) a.cur.dprev[s] = (T)dprev[id];
}

// first index (into xy, in points) of a coordinate pair that is not finite
// or lies outside the box; bad[0] must start above n
template <typename T>
__global__ void k_check_points(const T* xy, int32_t n, double x0, double y0, double x1, double y1, int32_t* bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = (double)xy[2 * i], y = (double)xy[2 * i + 1];
    if (!(x >= x0 && x <= x1 && y >= y0 && y <= y1)) atomicMin(bad, i);
}

template <typename T>
void launch_check_points(const T* xy, int32_t n, double x0, double y0, double x1, double y1, int32_t* bad,
                         cudaStream_t st) {
    int g = (n + kThreads - 1) / kThreads;
    if (g > 0) k_check_points<T><<<g, kThreads, 0, st>>>(xy, n, x0, y0, x1, y1, bad);
}
template void launch_check_points<double>(const double*, int32_t, double, double, double, double, int32_t*,
                                          cudaStream_t);
template void launch_check_points<float>(const float*, int32_t, double, double, double, double, int32_t*,
                                         cudaStream_t);

template <typename T>
void launch_set_state(const IterArgs<T>& a, int32_t s0, int32_t ns, const T* xy, const uint8_t* cls,
                      const double* dprev, cudaStream_t st) {
    int g = (ns + kThreads - 1) / kThreads;
    if (g > 0) k_set_state<T><<<g, kThreads, 0, st>>>(a, s0, ns, xy, cls, dprev);
}
template void launch_set_state<double>(const IterArgs<double>&, int32_t, int32_t, const double*, const uint8_t*,
                                       const double*, cudaStream_t);
template void launch_set_state<float>(const IterArgs<float>&, int32_t, int32_t, const float*, const uint8_t*,
                                      const double*, cudaStream_t);

template <typename T>
__global__ void k_get_state(const __grid_constant__ IterArgs<T> a, int32_t s0, int32_t ns, T* xy, uint8_t* cls,
                            double* dprev) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    s += s0;
    size_t id = (size_t)(a.cur.id[s] - s0);
    if (xy) {
        xy[2 * id] = a.cur.x[s];
        xy[2 * id + 1] = a.cur.y[s];
    }
    if (cls) cls[id] = a.cur.cls[s];
    if (dprev) dprev[id] = (double)a.cur.dprev[s];
}

template <typename T>
void launch_get_state(const IterArgs<T>& a, int32_t s0, int32_t ns, T* xy, uint8_t* cls, double* dprev,
                      cudaStream_t st) {
    int g = (ns + kThreads - 1) / kThreads;
    if (g > 0) k_get_state<T><<<g, kThreads, 0, st>>>(a, s0, ns, xy, cls, dprev);
}
template void launch_get_state<double>(const IterArgs<double>&, int32_t, int32_t, double*, uint8_t*, double*,
                                       cudaStream_t);
template void launch_get_state<float>(const IterArgs<float>&, int32_t, int32_t, float*, uint8_t*, double*,
                                      cudaStream_t);

// ------------------------------------------------------------------ standalone a1
__global__ void k_count_raw(const double* x, const double* y, int32_t n, double x0, double y0, double ibsx,
                            double ibsy, int32_t nbx, int32_t nby, int32_t* key, int32_t* rank, int32_t* cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int bx = (int)floor((x[i] - x0) * ibsx), by = (int)floor((y[i] - y0) * ibsy);
    bx = bx < 0 ? 0 : (bx >= nbx ? nbx - 1 : bx);
    by = by < 0 ? 0 : (by >= nby ? nby - 1 : by);
    int k = by * nbx + bx;
    key[i] = k;
    rank[i] = atomicAdd(&cnt[k], 1);
}

__global__ void k_scatter_raw(int32_t n, const int32_t* key, const int32_t* rank, const int32_t* bstart,
                              int32_t* sorted_idx) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    sorted_idx[bstart[key[i]] + rank[i]] = i;
}

// scratch layout: key[n] | rank[n] | counts[nb] | scan tiles (<= 1024)
void launch_bucket_raw(const double* x, const double* y, int32_t n, double x0, double y0, double bsx, double bsy,
                       int32_t nbx, int32_t nby, int32_t* bstart, int32_t* sorted_idx, int32_t* scratch,
                       cudaStream_t st) {
    int nb = nbx * nby;
    int32_t* key = scratch;
    int32_t* rank = scratch + n;
    int32_t* cnt = scratch + 2 * (size_t)n;
    int32_t* tiles = cnt + nb;
    cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)nb, st);
    int g = (n + kThreads - 1) / kThreads;
    if (g > 0)
        k_count_raw<<<g, kThreads, 0, st>>>(x, y, n, x0, y0, 1.0 / bsx, 1.0 / bsy, nbx, nby, key, rank, cnt);
    launch_scan(cnt, bstart, nb, tiles, st);
    if (g > 0) k_scatter_raw<<<g, kThreads, 0, st>>>(n, key, rank, bstart, sorted_idx);
}

// ------------------------------------------------------------------ a1 without allocation
// Scratch of mesh_bucket_points_noalloc: a file-scope device array, so the
// entry point never allocates.  Every GPU that loads the library holds it
// (16 MiB) until the process exits.  In host code g_bucket_scratch names a
// host-side stand-in, not a device address: kernels receive the address
// resolved by cudaGetSymbolAddress below.
constexpr size_t kNoallocScratchInts = size_t(1) << 22;
static __device__ __align__(256) int32_t g_bucket_scratch[kNoallocScratchInts];

static std::mutex g_scratch_mu;
static int32_t* g_scratch_ptr[256];  // per device ordinal, resolved once

// set-up, once per device, with that device current
static int32_t* noalloc_scratch(int& rc) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) {
        rc = set_error(TRIME_ECUDA, "cudaGetDevice failed");
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bucket_scratch);
        if (e != cudaSuccess || !p) {
            rc = set_error(TRIME_ECUDA, "cudaGetSymbolAddress of the bucketing scratch failed");
            return nullptr;
        }
        g_scratch_ptr[dev] = static_cast<int32_t*>(p);
    }
    return g_scratch_ptr[dev];
}

}  // namespace trime

extern "C" int mesh_bucket_points_noalloc(const double* x, const double* y, int64_t n, double x0, double y0,
                                          double x1, double y1, int32_t nbx, int32_t nby, int32_t* bucket_start,
                                          int32_t* sorted_idx, void* cuda_stream) {
    using namespace trime;
    if (n < 0 || nbx < 1 || nby < 1) return set_error(TRIME_EINVAL, "n < 0 or empty bucket grid");
    if (!(x1 > x0) || !(y1 > y0)) return set_error(TRIME_EINVAL, "empty box");
    if (!bucket_start || (n > 0 && (!x || !y || !sorted_idx))) return set_error(TRIME_EINVAL, "NULL pointer");
    size_t nb = (size_t)nbx * (size_t)nby;
    size_t tiles = nb / 4096 + 1;
    size_t need = 2 * (size_t)n + nb + tiles;
    if ((int64_t)nbx * nby > (int64_t)4096 * 1024 || need > kNoallocScratchInts)
        return set_error(TRIME_EINVAL, "mesh_bucket_points_noalloc: 2*n + nbx*nby + nbx*nby/4096 + 1 must not exceed "
                                       "4194304 (its fixed 16 MiB scratch)");
    int rc = 0;
    int32_t* scratch = noalloc_scratch(rc);
    if (!scratch) return rc;
    launch_bucket_raw(x, y, (int32_t)n, x0, y0, (x1 - x0) / nbx, (y1 - y0) / nby, nbx, nby, bucket_start, sorted_idx,
                      scratch, (cudaStream_t)cuda_stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(TRIME_ECUDA, cudaGetErrorString(e));
    return TRIME_OK;
}
