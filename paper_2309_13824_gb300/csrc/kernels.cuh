// kernels.cuh -- argument blocks and launchers of the iteration's kernels.
//
// Data layout in HBM (N points, T = double or float positions):
//   cur.{x,y,id,cls,dprev}  per-point state written by the update kernel
//   srt.{x,y,id,cls,dprev}  the same state counting-sorted by bucket (a1);
//                           every later kernel of the iteration indexes by
//                           sorted slot, so neighbours are near in memory
//   srt.cell / srt.key      geometry cell and bucket of each sorted slot
//   ring[N][32] int32       cell edge labels, CCW: neighbour slot (>= 0) or a
//                           bounding line (< 0); one 128-byte row per cell
//   ring_n[N] u8, cellR[N]  edge count, conservative max vertex distance
//   vmask[N] u32            bit t: triangle (slot, ring[t], ring[t+1]) valid
#pragma once
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

template <typename T>
struct IterArgs {
    int32_t n;
    int32_t force;       // ignore the terminated flag (rebuild-only calls)
    DevParams P;
    DevGrid sdf, siz;
    // geometry grid on the SDF grid's cells
    const uint8_t* gcls;
    const double* gh;
    const double* ggeps;
    const uint8_t* gidist;  // Chebyshev distance to the nearest non-inner cell, capped
    State<T> cur, srt;
    int32_t* cell;     // [n] geometry cell of each sorted slot (fixed formula)
    int32_t* key;      // [n] bucket of each cur point
    int32_t* rank;     // [n] rank inside its bucket
    int32_t* skey;     // [n] bucket of each sorted slot
    uint8_t* dom;      // [n] sorted slot has an exact duplicate with a larger id
    int32_t* bcount;   // [nb] bucket counts
    int32_t* bstart;   // [nb + 1]
    int32_t* scan_tmp;
    int32_t* ring;
    uint8_t* ring_n;
    float* cellR;
    uint32_t* vmask;
    EmitPartial* ep;
    UpdatePartial* up;
    DevCtrl* ctrl;
    double* dbg;       // [8][n] by original id, written when P.debug
    int32_t* ovf_list; // [n] cells whose 16-lane clipping ran out of lanes
    float4* pf;        // [n] sorted positions as float pairs (xhi, xlo, yhi, ylo)
    float* pS;         // [n] octagon span S = fac_voro_bound * h of each sorted slot
};

// a1: counting sort
template <typename T> void launch_bucket(const IterArgs<T>& a, cudaStream_t st);
void launch_scan(const int32_t* in, int32_t* out, int32_t n, int32_t* tmp, cudaStream_t st);
// a2
template <typename T> void launch_voronoi(const IterArgs<T>& a, cudaStream_t st);
// a3/a4 + quality partials (a8) + Eq. 3 sums
template <typename T> void launch_emit(const IterArgs<T>& a, int nblocks, cudaStream_t st);
// a8 finalisation + hybrid / termination logic
void launch_stats_pre(DevCtrl* ctrl, const EmitPartial* ep, int nparts, int decide, int force, DevParams P,
                      cudaStream_t st);
// a5/a6/a7
template <typename T> void launch_update(const IterArgs<T>& a, int nblocks, cudaStream_t st);
void launch_stats_post(DevCtrl* ctrl, const UpdatePartial* up, int nparts, cudaStream_t st);
// output helpers
template <typename T> void launch_tri_count(const IterArgs<T>& a, int32_t* cnt, cudaStream_t st);
template <typename T> void launch_tri_write(const IterArgs<T>& a, const int32_t* off, int32_t* tri, cudaStream_t st);
template <typename T> void launch_unpermute(const IterArgs<T>& a, T* out_xy, cudaStream_t st);
template <typename T> void launch_set_state(const IterArgs<T>& a, const T* xy, const uint8_t* cls,
                                            const double* dprev, cudaStream_t st);
void launch_predicates(const double* pts, const int32_t* ids, int32_t nq, int32_t* o_out, int32_t* c_out,
                       cudaStream_t st);
// standalone a1 on raw arrays (mesh_bucket_points)
void launch_bucket_raw(const double* x, const double* y, int32_t n, double x0, double y0, double bsx, double bsy,
                       int32_t nbx, int32_t nby, int32_t* bstart, int32_t* sorted_idx, int32_t* scratch,
                       cudaStream_t st);

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
