// kernels.cuh -- argument blocks and launchers of the iteration's kernels.
//
// Data layout in HBM (N points, T = double or float positions):
//   cur.{x,y,id,cls,dprev}  per-point state written by the update kernel
//   srt.{x,y,id,cls,dprev}  the same state counting-sorted by bucket (a1);
//                           every later kernel of the iteration indexes by
//                           sorted slot, so neighbours are near in memory
//   srt.cell / srt.key      geometry cell and bucket of each sorted slot
//   ring[N][64] int32       cell edge labels, CCW: neighbour slot (>= 0) or a
//                           bounding line (< 0); one 256-byte row per cell
//   ring_n[N] u8, cellR[N]  edge count, conservative max vertex distance
//   vmask[N] u64            bit t: triangle (slot, ring[t], ring[t+1]) valid
#pragma once
#include <string>

#include "common.cuh"

namespace trime {

template <typename T>
struct State {
    T* x;
    T* y;
    int32_t* id;
    uint8_t* cls;
    T* dprev;
};

// Everything a kernel reads that belongs to one mesh.  A batch concatenates
// its meshes' slots, each mesh padded to whole chunks of kChunk slots, so a
// block of the emit / update kernels and a warp of the Voronoi kernel always
// work on one mesh.
constexpr int kChunk = 256;
constexpr int kChunkShift = 8;

struct MeshView {
    DevParams P;
    DevGrid sdf, siz;
    // geometry grid on the SDF grid's cells
    const uint8_t* gcls;
    const double* gh;
    const double* ggeps;
    const uint8_t* gidist;  // Chebyshev distance to the nearest non-inner cell, capped
    DevCtrl* ctrl;
    int32_t soff, n;        // first slot, number of points
    int32_t boff, nb;       // first bucket, buckets (a pad bucket follows them)
    int32_t c0, c1;         // chunks [c0, c1): the emit / update partials of this mesh
    int32_t npad;           // padding slots after the points
    int32_t pad0;
};

template <typename T>
struct IterArgs {
    int32_t n;         // slots (single mesh: points; batch: padded total)
    int32_t force;     // ignore the terminated flags (rebuild-only calls)
    int32_t nmesh;     // meshes in Vs (batched launches)
    int32_t nbtot;     // buckets in bcount / bstart, pad buckets included
    MeshView V;        // the mesh of single-mesh launches
    const MeshView* Vs;     // [nmesh] per-mesh views of batched launches
    const int32_t* cmesh;   // [n / kChunk] mesh of each chunk
    int32_t* ovf_n;    // [4] cells queued for the 32-lane, the serial, the big-cell and the 16-lane Voronoi pass
    State<T> cur, srt;
    State<T> wrk;      // the positions a DistMesh iteration without re-triangulation moves (slot order)
    int32_t* cell;     // [n] geometry cell of each sorted slot (fixed formula)
    int32_t* key;      // [n] bucket of each cur point
    int32_t* rank;     // [n] provisional rank inside its bucket (atomics)
    int32_t* sidx;     // [n] point indices listed by bucket (provisional order inside a bucket)
    int32_t* skey;     // [n] bucket of each sorted slot
    uint8_t* dom;      // [n] sorted slot has an exact duplicate with a larger id
    int32_t* bcount;   // [nbtot] bucket counts
    int32_t* bstart;   // [nbtot + 1]
    int32_t* scan_tmp;
    int32_t* ring;
    uint8_t* ring_n;
    int32_t* warm;     // [n * kWarm] a slot's bisector neighbours at the last rebuild (-1 padded): old slots
                       // after the scatter, this rebuild's slots after k_dups
    int32_t* perm;     // [n] new slot of each old slot (written by the scatter)
    float* cellR;
    uint64_t* vmask;
    EmitPartial* ep;   // [n / kThreads] one per block of the emit kernel
    UpdatePartial* up;
    double* dbg;       // [8][n] by original id, written when P.debug
    int32_t* ovf0_list; // [n] cells whose 8-lane clipping ran out of lanes
    int32_t* ovf_list; // [n] cells whose 16-lane clipping ran out of lanes
    int32_t* ovf2_list; // [n] cells whose 32-lane clipping ran out of lanes (serial pass)
    int32_t* ovf3_list; // [n] cells with more edges than a ring row (big-cell pass on request)
    float4* pf;        // [n] sorted positions as float pairs (xhi, xlo, yhi, ylo)
    float2* pf3;       // [n] third parts: x = xhi + xlo + x3 exactly (FP64 positions)
    float* pS;         // [n] octagon span S = fac_voro_bound * h of each sorted slot
};

// the rebuild kernels of an iteration run unless the mesh has terminated or
// keeps its last triangulation (a forced rebuild always runs)
__device__ __forceinline__ bool skip_rebuild(const DevCtrl* c, int force) {
    return !force && (c->terminated || !c->retri);
}

// the mesh owning a slot: the launch's own view, or the batch table entry of
// the slot's chunk
template <bool B, typename T>
__device__ __forceinline__ const MeshView& mesh_of(const IterArgs<T>& a, int slot) {
    if constexpr (B) return a.Vs[__ldg(a.cmesh + (slot >> kChunkShift))];
    else return a.V;
}

// a1: counting sort
template <typename T> void launch_bucket(const IterArgs<T>& a, cudaStream_t st);
void launch_scan(const int32_t* in, int32_t* out, int32_t n, int32_t* tmp, cudaStream_t st);
// a2
template <typename T, bool B> void launch_voronoi_impl(const IterArgs<T>& a, int lanes, cudaStream_t st);
template <typename T>
inline void launch_voronoi(const IterArgs<T>& a, int lanes, cudaStream_t st) {
    if (a.Vs) launch_voronoi_impl<T, true>(a, lanes, st);
    else launch_voronoi_impl<T, false>(a, lanes, st);
}
// the cells listed in ovf3_list (more than kRingCap edges) rebuilt into
// rings of up to 1024 edges (single mesh): scratch (1024 + 97) float4 per
// cell, rings 1024 int32 per cell, lens one per cell
template <typename T>
void launch_voronoi_big(const IterArgs<T>& a, int32_t n, float4* scratch, int32_t* rings, int32_t* lens,
                        cudaStream_t st);
constexpr int kBigRing = 1024;
constexpr size_t kBigScratchF4 = (size_t)kBigRing + 1 + 96;
// medial points of the big cells: emission decided by the fixed formulas
template <typename T>
void launch_medial_big(const IterArgs<T>& a, int32_t n, const int32_t* rings, const int32_t* lens, double* v,
                       uint8_t* flags, cudaStream_t st);
// a3/a4 + quality partials (a8) + Eq. 3 sums
template <typename T> void launch_emit(const IterArgs<T>& a, int nblocks, cudaStream_t st);
// a DistMesh iteration that keeps the last triangulation (Algorithm 1): the
// current positions into wrk and the Eq. 3 sums over the kept valid edges
template <typename T> void launch_dm_keep(const IterArgs<T>& a, int nblocks, cudaStream_t st);
// a8 finalisation + hybrid / termination logic
template <typename T> void launch_stats_pre(const IterArgs<T>& a, int decide, cudaStream_t st);
// a5/a6/a7
template <typename T> void launch_update(const IterArgs<T>& a, int nblocks, cudaStream_t st);
template <typename T> void launch_stats_post(const IterArgs<T>& a, cudaStream_t st);
// point addition (Sec. 3.6, 3.7) on a paused single mesh of n0 points whose
// ntri valid triangles have owner offsets toff: keys (kAddKeyBytes per
// triangle), selection of nadd, per-owner counts and offsets by id (cnt_id,
// off_id: n0 + 1 each), geometry rescaling and the new points at slots
// [n0, n0 + nadd) of cur; hist is 256 device ints, hhist 256 pinned host ints
constexpr size_t kAddKeyBytes = 24;
template <typename T>
int add_select(const IterArgs<T>& a, int32_t n0, int32_t ntri, int64_t nadd, const int32_t* toff, void* keys,
               int32_t* hist, int32_t* hhist, int32_t* cnt_id, int32_t* off_id, int32_t* scan_tmp, double* gh,
               double* ggeps, int32_t nc, double scale, cudaStream_t st, std::string& err);
// Sec. 3.5 initial points: point q uniform in cell pcell[q] (SplitMix64
// stream of `seed`), projected by damped Newton when outside a boundary cell
void launch_init_points(const DevGrid& sdf, const uint8_t* gcls, const double* ggeps, const int32_t* pcell,
                        int64_t n, uint64_t seed, double damping, int newton_max, double* out, cudaStream_t st);
// medial points (Sec. 3.3) of the ns points of a single mesh from its last
// triangulation, by id: v[4 id ..] = (v1, v2), flags bit 0 / 1 = present
template <typename T> void launch_medial(const IterArgs<T>& a, int32_t ns, double* v, uint8_t* flags,
                                         cudaStream_t st);
// output helpers on the slots [s0, s0 + ns) of one mesh whose ids start at s0
template <typename T> void launch_tri_count(const IterArgs<T>& a, int32_t s0, int32_t ns, int32_t* cnt,
                                            cudaStream_t st);
template <typename T> void launch_tri_write(const IterArgs<T>& a, int32_t s0, int32_t ns, const int32_t* off,
                                            int32_t* tri, cudaStream_t st);
template <typename T> void launch_unpermute(const IterArgs<T>& a, int32_t s0, int32_t ns, T* out_xy,
                                            cudaStream_t st);
template <typename T> void launch_set_state(const IterArgs<T>& a, int32_t s0, int32_t ns, const T* xy,
                                            const uint8_t* cls, const double* dprev, cudaStream_t st);
template <typename T> void launch_check_points(const T* xy, int32_t n, double x0, double y0, double x1, double y1,
                                               int32_t* bad, cudaStream_t st);
template <typename T> void launch_get_state(const IterArgs<T>& a, int32_t s0, int32_t ns, T* xy, uint8_t* cls,
                                            double* dprev, cudaStream_t st);
void launch_predicates(const double* pts, const int32_t* ids, int32_t nq, int32_t* o_out, int32_t* c_out,
                       cudaStream_t st);
// standalone a1 on raw arrays (mesh_bucket_points)
void launch_bucket_raw(const double* x, const double* y, int32_t n, double x0, double y0, double bsx, double bsy,
                       int32_t nbx, int32_t nby, int32_t* bstart, int32_t* sorted_idx, int32_t* scratch,
                       cudaStream_t st);

// ------------------------------------------------------------------ learned model
constexpr int kMlpFeat = 39;   // features in use
constexpr int kMlpIn = 48;     // padded input width (a multiple of 16)
constexpr int kMlpHid = 64;
constexpr int kMlpOut = 2;
constexpr int kMlpOutPad = 16;
// flat FP32 parameter vector: W1 (64 x 48), b1, W2 (64 x 64), b2, W3 (2 x 64), b3
constexpr int kOW1 = 0, kOB1 = kOW1 + kMlpHid * kMlpIn, kOW2 = kOB1 + kMlpHid, kOB2 = kOW2 + kMlpHid * kMlpHid,
              kOW3 = kOB2 + kMlpHid, kOB3 = kOW3 + kMlpOut * kMlpHid, kMlpParams = kOB3 + kMlpOut;

struct MlpDev {
    const float* p;        // FP32 parameters
    const uint16_t* w1;    // BF16 copies: W1 (64 x 48), W2 (64 x 64), W3 (16 x 64, rows >= 2 zero)
    const uint16_t* w2;
    const uint16_t* w3;
};

// Y[i] (2 floats) for the rows X[idx ? idx[i] : i] (48 BF16 each), i < n
void launch_mlp_forward(const MlpDev& w, const uint16_t* X, const int32_t* idx, int n, float* Y, int* err,
                        cudaStream_t st);
// d/dp of sum (Y - T)^2 * scale / 2 over the n rows, as per-CTA partial sums
// in gpart[c][kMlpParams] for c < the returned count (at most kGradParts);
// loss += that sum
constexpr int kGradParts = 152;
int launch_mlp_grad(const MlpDev& w, const uint16_t* X, const float* T, const int32_t* idx, int n, float scale,
                    float* gpart, double* loss, int* err, cudaStream_t st);
// features of every slot of a single mesh (slot order, or by point id with
// by_id), h_i per row, optionally the positions by id; the last move is the
// position minus (qx, qy)[id] (zero without them)
template <typename T>
void launch_features(const IterArgs<T>& a, uint16_t* X, float* H, T* px, T* py, const T* qx, const T* qy, int by_id,
                     float method_cvd, cudaStream_t st);
// (qx, qy)[id] = the current positions (cur)
template <typename T>
void launch_snapshot(const IterArgs<T>& a, T* qx, T* qy, cudaStream_t st);
// moves cur <- srt + h_i * Y (slot order), clamped to jump * fac_pt * h_i, treated as Sec. 4.3
template <typename T>
void launch_propose(const IterArgs<T>& a, const float* Y, float jump, cudaStream_t st);
// T[id] = (cur position - (px, py)[id]) / H[id]
template <typename T>
void launch_targets(const IterArgs<T>& a, const T* px, const T* py, const float* H, float* Tout, cudaStream_t st);

// the quality report of the slots [s0, s0 + ns) of one mesh's last rebuild
// (quality.cu): device scratch for counts, offsets, per-triangle and
// per-edge values (cap_t triangles, cap_e edges), block partials and a
// 256-bin histogram with its pinned host copy
struct QPartial;
}  // namespace trime
struct mesh_quality_stats;  // include/trime.h
namespace trime {
struct QBufs {
    int32_t *tcnt, *ecnt, *toff, *eoff, *scan_tmp;
    double *alpha, *beta, *ang, *dev;
    QPartial* part;
    unsigned int* hist;
    unsigned int* hhist;
};
template <typename T>
int quality_report(const IterArgs<T>& a, int32_t s0, int32_t ns, double fac_mu, const QBufs& b, int64_t cap_t,
                   int64_t cap_e, cudaStream_t st, ::mesh_quality_stats* q, std::string& err);

// records the calling thread's error message (mesh_last_error) and returns code
int set_error(int code, const char* msg);

constexpr int kThreads = 256;
constexpr int kVoroThreads = 128;

// bucket of a point: float arithmetic, clamped; the count kernel and the
// Voronoi kernel call this same function so assignments agree
template <typename T>
__device__ __forceinline__ void bucket_of(const DevParams& P, T x, T y, int& bx, int& by) {
    float fx = ((float)x - P.bx0f) * P.ibsxf;
    float fy = ((float)y - P.by0f) * P.ibsyf;
    bx = (int)floorf(fx);
    by = (int)floorf(fy);
    bx = bx < 0 ? 0 : (bx >= P.nbx ? P.nbx - 1 : bx);
    by = by < 0 ? 0 : (by >= P.nby ? P.nby - 1 : by);
}

}  // namespace trime
