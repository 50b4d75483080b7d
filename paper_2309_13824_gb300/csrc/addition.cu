// addition.cu -- the point-addition scheme of TriMe++ Sec. 3.6 and the
// rescaled quantities of Sec. 3.7: the kernels the host runs while an
// iteration has paused the graph for an addition (ctrl->terminated == 2;
// single mesh, slots [0, n0), the triangulation of that iteration in
// ring / vmask / srt).
//
// Selection is exact and needs no sort.  Every valid triangle, counted once
// by its smallest-id vertex (its owner) in ring order, gets a 20-byte key:
// the complemented bits of its FP64 ratio R_circ / h_i (larger ratio first;
// h_i of the geometry cell holding the centroid), then its vertex ids in
// ascending order.  The keys are distinct, so "the N_add smallest keys" is a
// well-defined set; a most-significant-byte-first radix select finds the
// shortest key prefix whose keys at or below it are exactly those (one
// 256-bin histogram per byte, read by the host, stopping at the first byte
// whose bin is taken whole).  New points are numbered in the ascending order
// of their triangles' vertex triples: the triple starts with the owner's id,
// so an exclusive prefix sum of the per-owner counts in id order plus the
// rank of the triangle's (b, c) pair among its owner's selected triangles
// numbers them without sorting.
#include <algorithm>
#include <cstring>
#include <string>

#include "kernels.cuh"

namespace trime {

// a key as three big-endian words; bytes 20..23 are zero
struct AddKey {
    unsigned long long w0, w1, w2;
};

// the first nbytes bytes of the key as words (the rest zero)
struct AddPrefix {
    unsigned long long t0, t1, t2;
    int32_t nbytes;
    int32_t pad;
};

__device__ __forceinline__ unsigned long long prefix_mask(int nbytes, int word) {
    int b = nbytes - 8 * word;
    if (b <= 0) return 0ull;
    if (b >= 8) return ~0ull;
    return ~0ull << (64 - 8 * b);
}

__device__ __forceinline__ int key_byte(const AddKey& k, int p) {
    unsigned long long w = p < 8 ? k.w0 : (p < 16 ? k.w1 : k.w2);
    return (int)((w >> (56 - 8 * (p & 7))) & 0xFFull);
}

__device__ __forceinline__ bool prefix_eq(const AddKey& k, const AddPrefix& q) {
    return (k.w0 & prefix_mask(q.nbytes, 0)) == q.t0 && (k.w1 & prefix_mask(q.nbytes, 1)) == q.t1 &&
           (k.w2 & prefix_mask(q.nbytes, 2)) == q.t2;
}

// the key's first q.nbytes bytes are at or below the prefix: the key is selected
__device__ __forceinline__ bool prefix_le(const AddKey& k, const AddPrefix& q) {
    unsigned long long a0 = k.w0 & prefix_mask(q.nbytes, 0), a1 = k.w1 & prefix_mask(q.nbytes, 1),
                       a2 = k.w2 & prefix_mask(q.nbytes, 2);
    if (a0 != q.t0) return a0 < q.t0;
    if (a1 != q.t1) return a1 < q.t1;
    return a2 <= q.t2;
}

// the owned valid triangles of slot s, in ring order: f(j, k) with j, k the
// other two slots, (s, j, k) counter-clockwise
template <typename T, typename F>
__device__ __forceinline__ void for_owned(const IterArgs<T>& a, int s, F&& f) {
    int ne = a.ring_n[s];
    uint64_t vm = a.vmask[s];
    int idi = a.srt.id[s];
    for (int t = 0; t < ne; t++) {
        if (!((vm >> t) & 1ull)) continue;
        int j = a.ring[(size_t)s * kRingCap + t], k = a.ring[(size_t)s * kRingCap + (t + 1 == ne ? 0 : t + 1)];
        if (idi < a.srt.id[j] && idi < a.srt.id[k]) f(j, k);
    }
}

template <typename T>
__device__ __forceinline__ void centroid_fixed(const IterArgs<T>& a, int s, int j, int k, double& gx, double& gy) {
    gx = fdiv(fadd(fadd((double)a.srt.x[s], (double)a.srt.x[j]), (double)a.srt.x[k]), 3.0);
    gy = fdiv(fadd(fadd((double)a.srt.y[s], (double)a.srt.y[j]), (double)a.srt.y[k]), 3.0);
}

// one thread per owner slot: the keys of its owned triangles at off[s] ...
template <typename T>
__global__ void __launch_bounds__(kThreads) k_add_keys(const __grid_constant__ IterArgs<T> a, int32_t n0,
                                                       const int32_t* off, AddKey* keys) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n0) return;
    const MeshView& V = a.V;
    int ncx = V.sdf.nx - 1;
    int o = off[s];
    int idi = a.srt.id[s];
    double xi = (double)a.srt.x[s], yi = (double)a.srt.y[s];
    for_owned(a, s, [&](int j, int k) {
        double ox, oy, R;
        circumcentre_fixed(xi, yi, (double)a.srt.x[j], (double)a.srt.y[j], (double)a.srt.x[k], (double)a.srt.y[k],
                           ox, oy, R);
        double gx, gy;
        centroid_fixed(a, s, j, k, gx, gy);
        int gi, gj;
        point_cell_fixed(V.sdf, gx, gy, gi, gj);
        double r = fdiv(R, V.gh[gj * ncx + gi]);
        if (!(r > 0.0)) r = 0.0;  // a NaN ratio ranks last
        int idj = a.srt.id[j], idk = a.srt.id[k];
        unsigned lo = (unsigned)min(idj, idk), hi = (unsigned)max(idj, idk);
        AddKey K;
        K.w0 = ~(unsigned long long)__double_as_longlong(r);
        K.w1 = ((unsigned long long)(unsigned)idi << 32) | lo;
        K.w2 = (unsigned long long)hi << 32;
        keys[o++] = K;
    });
}

// histogram of byte q.nbytes over the keys that match the prefix
__global__ void __launch_bounds__(256) k_add_hist(const AddKey* keys, int32_t n, AddPrefix q, int32_t* hist) {
    __shared__ int sh[256];
    sh[threadIdx.x] = 0;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        AddKey k = keys[i];
        if (prefix_eq(k, q)) atomicAdd(&sh[key_byte(k, q.nbytes)], 1);
    }
    __syncthreads();
    if (sh[threadIdx.x]) atomicAdd(&hist[threadIdx.x], sh[threadIdx.x]);
}

// selected triangles per owner, written at the owner's id
template <typename T>
__global__ void __launch_bounds__(kThreads) k_add_count(const __grid_constant__ IterArgs<T> a, int32_t n0,
                                                        const int32_t* off, const AddKey* keys, AddPrefix q,
                                                        int32_t* cnt_id) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n0) return;
    int c = 0;
    for (int o = off[s]; o < off[s + 1]; o++) c += prefix_le(keys[o], q) ? 1 : 0;
    cnt_id[a.srt.id[s]] = c;
}

// geometry quantities times s (Sec. 3.7)
__global__ void k_scale_geometry(double* gh, double* ggeps, int32_t nc, double s) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    gh[c] = fmul(gh[c], s);
    ggeps[c] = fmul(ggeps[c], s);
}

// class of a new point by the rule for initial points (Sec. 4.3 classes, a
// point outside counting as boundary), fixed formulas
__device__ __forceinline__ uint8_t initial_class(const MeshView& V, double x, double y) {
    int gi, gj;
    if (!point_cell_fixed(V.sdf, x, y, gi, gj)) return PT_BOUNDARY;
    int c = gj * (V.sdf.nx - 1) + gi;
    uint8_t k = V.gcls[c];
    if (k == CELL_INNER) return PT_INNER;
    if (k == CELL_OUTER) return PT_BOUNDARY;
    double sd = bilin_fixed(V.sdf, x, y), g = V.ggeps[c];
    if (fabs(sd) <= g) return PT_BOUNDARY;
    return sd < -g ? PT_INNER : PT_BOUNDARY;
}

// one thread per owner slot: its selected triangles' centroids become points
// n0 + off_id[owner id] + rank of (b, c) among the owner's selected triangles;
// a single mesh's slot of id i is i.  Reads the rescaled geometry.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_add_write(const __grid_constant__ IterArgs<T> a, int32_t n0,
                                                        const int32_t* off, const AddKey* keys, AddPrefix q,
                                                        const int32_t* off_id) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n0) return;
    const MeshView& V = a.V;
    int o0 = off[s], o1 = off[s + 1];
    int base = off_id[a.srt.id[s]];
    int o = o0;
    for_owned(a, s, [&](int j, int k) {
        AddKey K = keys[o];
        o++;
        if (!prefix_le(K, q)) return;
        int rank = 0;
        for (int u = o0; u < o1; u++) {
            AddKey L = keys[u];
            if (prefix_le(L, q) && (L.w1 < K.w1 || (L.w1 == K.w1 && L.w2 < K.w2))) rank++;
        }
        double gx, gy;
        centroid_fixed(a, s, j, k, gx, gy);
        T px = (T)gx, py = (T)gy;
        int nid = n0 + base + rank;
        a.cur.x[nid] = px;
        a.cur.y[nid] = py;
        a.cur.id[nid] = nid;
        a.cur.cls[nid] = initial_class(V, (double)px, (double)py);
        int gi, gj;
        point_cell_fixed(V.sdf, (double)px, (double)py, gi, gj);
        a.cur.dprev[nid] = (T)V.gh[gj * (V.sdf.nx - 1) + gi];  // a first move of h_i
        // the triangle's corners are the new point's first clipping candidates
        int32_t* row = a.ring + (size_t)nid * kRingCap;
        row[0] = s;
        row[1] = j;
        row[2] = k;
        a.ring_n[nid] = 3;
    });
}

// ------------------------------------------------------------------ host side
// keys, radix select, per-owner counts and their prefix sum, the rescaling
// by `scale` and the new points; the host reads one histogram per key byte.
// Returns 0, or -1 (CUDA error) / -2 (inconsistent keys) with a message.
template <typename T>
int add_select(const IterArgs<T>& a, int32_t n0, int32_t ntri, int64_t nadd, const int32_t* toff, void* keys_v,
               int32_t* hist, int32_t* hhist, int32_t* cnt_id, int32_t* off_id, int32_t* scan_tmp, double* gh,
               double* ggeps, int32_t nc, double scale, cudaStream_t st, std::string& err) {
    auto cuda_fail = [&](const char* what) {
        err = std::string(what) + ": " + cudaGetErrorString(cudaGetLastError());
        return -1;
    };
    AddKey* keys = static_cast<AddKey*>(keys_v);
    int g = (n0 + kThreads - 1) / kThreads;
    k_add_keys<T><<<g, kThreads, 0, st>>>(a, n0, toff, keys);
    AddPrefix q;
    std::memset(&q, 0, sizeof q);
    int64_t need = nadd;
    int hb = std::max(1, std::min(1216, (ntri + 255) / 256));
    bool done = false;
    for (int p = 0; p < 20 && !done; p++) {
        q.nbytes = p;
        if (cudaMemsetAsync(hist, 0, 256 * sizeof(int32_t), st) != cudaSuccess) return cuda_fail("selection memset");
        k_add_hist<<<hb, 256, 0, st>>>(keys, ntri, q, hist);
        if (cudaMemcpyAsync(hhist, hist, 256 * sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return cuda_fail("selection histogram");
        int64_t cum = 0;
        int b = 0;
        for (; b < 256; b++) {
            if (cum + hhist[b] >= need) break;
            cum += hhist[b];
        }
        if (b == 256) {
            err = "point addition: fewer triangle keys than points to add";
            return -2;
        }
        unsigned long long bits = (unsigned long long)b << (56 - 8 * (p & 7));
        if (p < 8) q.t0 |= bits;
        else if (p < 16) q.t1 |= bits;
        else q.t2 |= bits;
        need -= cum;
        q.nbytes = p + 1;
        done = hhist[b] == need;
    }
    if (!done) {
        err = "point addition: two triangles with the same key";
        return -2;
    }
    k_add_count<T><<<g, kThreads, 0, st>>>(a, n0, toff, keys, q, cnt_id);
    launch_scan(cnt_id, off_id, n0, scan_tmp, st);
    if (nc > 0) k_scale_geometry<<<(nc + 255) / 256, 256, 0, st>>>(gh, ggeps, nc, scale);
    k_add_write<T><<<g, kThreads, 0, st>>>(a, n0, toff, keys, q, off_id);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail("point addition");
    return 0;
}

template int add_select<double>(const IterArgs<double>&, int32_t, int32_t, int64_t, const int32_t*, void*, int32_t*,
                                int32_t*, int32_t*, int32_t*, int32_t*, double*, double*, int32_t, double,
                                cudaStream_t, std::string&);
template int add_select<float>(const IterArgs<float>&, int32_t, int32_t, int64_t, const int32_t*, void*, int32_t*,
                               int32_t*, int32_t*, int32_t*, int32_t*, double*, double*, int32_t, double,
                               cudaStream_t, std::string&);

}  // namespace trime
