/*
 * trime.h -- C ABI of the GB300 meshing-iteration library.
 *
 * One meshing iteration of TriMe++ (Lu & Rycroft, arXiv 2309.13824) on one
 * GPU: bucket the points into a uniform grid, build every point's bounded
 * Voronoi cell by half-plane clipping, read the Delaunay triangles off the
 * cells and keep the valid ones, then move the points (DistMesh springs, CVD
 * centroids or the hybrid of the two) and project escaped points back through
 * the bilinear signed-distance grid.
 *
 * Conventions shared by every entry point:
 *  - Return value: 0 on success, a negative TRIME_E* code on failure; the
 *    message of the last failure on the calling thread is mesh_last_error().
 *  - Ownership: the library deep-copies every input at mesh_init and owns all
 *    device memory it allocates; output functions copy into caller buffers.
 *  - Streams: every call is ordered on the stream given at mesh_init.  Calls
 *    that return data to the host synchronise that stream.
 *  - No torch types cross this boundary: plain pointers and sizes only.
 */
#ifndef TRIME_H
#define TRIME_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TRIME_OK 0
#define TRIME_EINVAL (-1)     /* bad argument (null pointer, size, non-finite value) */
#define TRIME_ENOMEM (-2)     /* device or host allocation failed                   */
#define TRIME_ECUDA (-3)      /* a CUDA runtime call failed                          */
#define TRIME_ECAPACITY (-4)  /* output buffer too small; *n_out holds the size needed */
#define TRIME_ETIMEOUT (-5)   /* a bounded device wait ran out                       */
#define TRIME_EDEVICE (-6)    /* the device reported an error (see mesh_stats counters) */

/* A node-centred grid sampled bilinearly: node (i,j) sits at
 * (x0 + i*(x1-x0)/(nx-1), y0 + j*(y1-y0)/(ny-1)); values are row-major
 * v[j*nx + i] in HOST memory (float32).  nx, ny >= 2.  Used for the signed
 * distance field (Sec. 3.1: negative inside, positive outside) and for the
 * element sizing field mu (Sec. 3.3, Eq. 7; density rho = 1/mu^2, Eq. 8). */
typedef struct {
    int32_t nx, ny;
    double x0, y0, x1, y1;
    const float* v;
} mesh_grid2d;

/* Control parameters; mesh_default_params fills the paper's App. B defaults.
 * Fields the paper leaves open carry the readings stated beside them. */
typedef struct {
    int32_t precision;       /* 0: FP64 positions; 1: FP32 positions, FP64 predicates   */
    int32_t method;          /* 0 DistMesh (Sec. 2.2), 1 CVD (Sec. 2.3), 2 hybrid (Sec. 2.4) */
    int32_t bounded;         /* 1: octagon cell bound of span S = fac_voro_bound*h (Sec. 4.1) */
    int32_t validity;        /* 1: keep only triangles passing Tests 1-3 (Sec. 4.1)     */
    int32_t newton_max;      /* Newton steps of the point projection, T_ct^newton = 10  */
    int32_t trace_max;       /* sphere-trace steps (paper silent): 64                   */
    int32_t quad_max_level;  /* centroid quadrature level cap (paper silent): 8         */
    int32_t debug;           /* 1: mesh_step records per-point moves for mesh_get_debug */
    double fac_F;            /* 1.2   desired-length factor (Eq. 3)                       */
    double k_spring;         /* 1.0   spring stiffness k (paper lists none)               */
    double dt;               /* 0.2   forward-Euler step (paper lists none)               */
    double fac_pt;           /* 0.4   movement clamp T_pt = fac_pt*h_i (Sec. 3.7)          */
    double fac_geps;         /* 0.01  geps_i = fac_geps*min(h_i, h_avg)                    */
    double fac_voro_bound;   /* 5     octagon span factor                                  */
    double fac_end;          /* 0.001 small-movement factor                                */
    double T_circ;           /* 0.4   circumcentre test threshold (Test 3)                 */
    double T_switch;         /* 0.0015 hybrid switch threshold                             */
    double T_end_q;          /* 0.001 quality termination threshold                        */
    double T_end_amax;       /* 0.005 max-aspect-ratio termination threshold               */
    double N_opt;            /* 3.3   points per bucket of the neighbour grid (Sec. 3.2)   */
    double eta;              /* 0.5   selected-boundary band factor (Sec. 3.5)             */
    double damping;          /* 1.0   Newton damping alpha-hat                             */
    double fac_retria;       /* 0.1   DistMesh (method 0) re-triangulates only after some point
                                      moved more than fac_retria*h_i since the last triangulation
                                      (Algorithm 1); 0: every iteration                     */
    double fac_add;          /* 0.6   point addition: N_add = min(floor(fac_add*N_current),
                                      N_total - N_current), at least 1 (Sec. 3.6)          */
    double T_add;            /* 0.002 add points once the 1/2-means of alpha and beta both
                                      change by less than this (Sec. 3.6)                  */
    int64_t n_total;         /* 0     N_total: above mesh_init's n, the mesh starts with n
                                      points and grows to n_total by the point-addition
                                      scheme (Sec. 3.6); single meshes only                */
} mesh_params;

/* Statistics of the last iteration run by mesh_step (or of mesh_rebuild). */
typedef struct {
    int32_t iterations;        /* iterations executed by the call                         */
    int32_t terminated;        /* a termination criterion of Sec. 4 holds                 */
    int32_t method;            /* move of the last executed iteration: 0 DM, 1 CVD, -1 none */
    int32_t switched;          /* hybrid has switched to CVD                              */
    int64_t n_tri;             /* valid triangles of the last rebuild                     */
    int64_t n_edges;           /* unique valid edges                                      */
    double half_mean_alpha;    /* 1/2-mean of the aspect ratio alpha (Eqs. 11-12)         */
    double half_mean_beta;     /* 1/2-mean of the edge ratio beta                         */
    double max_alpha, max_beta;
    double min_angle_deg;
    double mean_size_dev;      /* mean |l / (fac_mu mu(m)) - 1| over valid edges          */
    double fac_mu;             /* Eq. 3 scaling factor                                    */
    int64_t exact_calls;       /* predicate evaluations that needed exact arithmetic      */
    int64_t clip_inconsistent; /* clips whose cut set was not one run (0 expected)        */
    int64_t ring_overflow;     /* cells with more than 64 edges (results dropped)         */
    int64_t exact_overflow;    /* exact-arithmetic capacity or underflow guard tripped    */
    int64_t newton_fail;       /* projections that kept p_old (Sec. 4.3)                  */
    int64_t trace_cap;         /* sphere traces that hit trace_max                        */
    int64_t quad_cap;          /* centroids that hit quad_max_level                       */
    int64_t dup_points;        /* points whose cell is empty (exact duplicate, SoS)       */
    int32_t small_moves;       /* every inner point moved less than fac_end*h_i           */
    int32_t target_reached;    /* stopped at the quality target (mesh_set_quality_target) */
    /* Voronoi work of the last call, counted only with mesh_params.debug = 1: */
    int64_t vor_candidates;    /* candidate points loaded within the security radius      */
    int64_t vor_picks;         /* candidates applied to a cell                            */
    int64_t vor_cuts;          /* applications that changed a cell                        */
    int64_t vor_rings;         /* bucket rings scanned (summed over cells)                */
    int64_t vor_wide;          /* cells queued for a wider Voronoi pass                  */
    int64_t triangulations;    /* iterations of the call that re-triangulated             */
    int64_t added;             /* points added by the call (Sec. 3.6)                     */
    int64_t n_points;          /* N_current after the call                                */
    /* more Voronoi work counters (mesh_params.debug = 1 only): */
    int64_t vor_fp64;          /* cut decisions the float filter left to the FP64 filter  */
    int64_t vor_resolve;       /* polygon vertices solved again in double                 */
    int64_t vor_direct;        /* cells built in one step from their previous neighbours  */
} mesh_stats;

/* Quality report of a mesh's last rebuild (mesh_quality): the statistics
 * the paper tabulates at termination (Sec. 5 tables: median, mean, maximum
 * and standard deviation of the aspect ratio alpha = R_circ / (2 R_in) and
 * the edge ratio beta = l_max / l_min of the valid triangles (Sec. 3.6 Eqs.
 * 11-12), the shares with alpha < 1.2 and < 2), the minimum angle, a
 * histogram of alpha, and the deviation of the valid edges' lengths from the
 * sizing field, |l / (fac_mu mu(m)) - 1| with Eq. 3's fac_mu.  All in FP64
 * at the positions that rebuild triangulated. */
typedef struct mesh_quality_stats {
    int64_t n_tri;             /* valid triangles                                        */
    int64_t n_edges;           /* valid edges                                            */
    double median_alpha;       /* lower median: rank floor((n - 1) / 2) of the sorted values */
    double median_beta;
    double mean_alpha, mean_beta;
    double max_alpha, max_beta;
    double std_alpha, std_beta;       /* population standard deviations               */
    double frac_alpha_lt_1_2;  /* share of the triangles with alpha < 1.2                */
    double frac_alpha_lt_2;    /* share with alpha < 2                                   */
    double min_angle_deg;
    int64_t alpha_hist[10];    /* triangles per alpha bin; bin k holds [e_k, e_{k+1}) with
                                  e = 1, 1.05, 1.1, 1.2, 1.3, 1.5, 2, 3, 5, 10, +inf
                                  (a value rounded below 1 counts in bin 0)            */
    double fac_mu;             /* Eq. 3 factor of the rebuild                            */
    double mean_size_dev;      /* mean of |l / (fac_mu mu(m)) - 1| over the valid edges  */
    double p95_size_dev;       /* its 95th percentile (nearest rank: rank ceil(0.95 n))  */
} mesh_quality_stats;

typedef struct mesh_s mesh_t;

/* Fill *p with the defaults listed above.  Never fails. */
void mesh_default_params(mesh_params* p);

/* Create a mesh on the current CUDA device.
 *  sdf, sizing: host grids, deep-copied (sizing values must be > 0).
 *  xy: HOST array of n (x, y) pairs, float64 if p->precision == 0 else
 *      float32, every point finite and inside the SDF grid's box.
 *  n >= 0.  p may be NULL for the defaults.  cuda_stream: a cudaStream_t
 *  (NULL = legacy default stream) on which all later work is ordered.
 * Precomputes the geometry grid on the SDF grid's cells (Sec. 3.2 classes,
 * Sec. 3.7 h_i and geps_i, h_i from N_current = n), allocates all device
 * buffers (for max(n, p->n_total) points) and captures one iteration into a
 * CUDA graph.  Errors: TRIME_EINVAL, TRIME_ENOMEM, TRIME_ECUDA. */
int mesh_init(mesh_t** out, const mesh_grid2d* sdf, const mesh_grid2d* sizing, const void* xy, int64_t n,
              const mesh_params* p, void* cuda_stream);

/* Procedure I (Sec. 2.1, 4.1) at the current positions: cells, triangles,
 * Tests 1-3 and quality, without moving.  Synchronises; fills *stats if given. */
int mesh_rebuild(mesh_t* m, mesh_stats* stats);

/* Run up to n_iters meshing iterations (Algorithms 1-2; hybrid Sec. 4.2),
 * each one graph launch: rebuild, quality, hybrid/termination decision, move,
 * point treatment (Sec. 4.3).  Once a termination criterion of Sec. 4 holds
 * the later iterations are device-side no-ops.  With stats != NULL the host
 * also checks for termination every 32 iterations (and stops launching),
 * synchronises at the end, fills *stats and returns TRIME_EDEVICE if a
 * capacity guard tripped.  With stats == NULL (and no point addition pending,
 * below) the call only enqueues the n_iters launches on the caller's stream
 * and never waits for the device.
 * While N_current < N_total (point addition, Sec. 3.6) the hybrid switch and
 * the termination tests are not evaluated; an iteration whose 1/2-means of
 * alpha and beta both changed by less than T_add since the previous one
 * (never measured across an addition) does not move: it pauses the graph
 * and the host adds N_add points at the centroids of the valid triangles
 * with the largest R_circ/h_i (h_i at the centroid; ties to the smaller
 * ascending vertex-index triple), numbered N_current, N_current+1, ... in the
 * ascending order of those triples, multiplies h_i, geps_i and h_avg by
 * sqrt(N_old/N_current) (Sec. 3.7), classifies the new points like initial
 * points and re-captures the iteration for the new size.  Such calls check
 * for a pause every 8 iterations and synchronise even with stats == NULL;
 * n_iters counts executed iterations (an addition is one). */
int mesh_step(mesh_t* m, int32_t n_iters, mesh_stats* stats);

/* N_current and N_total of a mesh (host-side state; no synchronisation). */
int mesh_get_count(mesh_t* m, int64_t* n_current, int64_t* n_total);

/* The quality report of the last rebuild (of mesh_rebuild, or of the last
 * iteration of mesh_step that re-triangulated; after mesh_set_state or an
 * addition a rebuild runs first), into *q.  The per-triangle and per-edge
 * values are computed on the device; medians and the percentile are exact
 * order statistics.  Synchronous.  Errors: TRIME_EINVAL, TRIME_ENOMEM,
 * TRIME_ECUDA. */
int mesh_quality(mesh_t* m, mesh_quality_stats* q);

/* Valid triangles of the last rebuild as int32 (a, b, c) point indices, a the
 * smallest index, counter-clockwise; order unspecified.  tri may be host or
 * device memory (detected); cap in triangles.  If cap is too small returns
 * TRIME_ECAPACITY with *n_out = the number needed. */
int mesh_get_triangles(mesh_t* m, int32_t* tri, int64_t cap, int64_t* n_out);

/* Current positions in input order, float64 or float32 as the precision;
 * host or device buffer of cap points. */
int mesh_get_points(mesh_t* m, void* xy, int64_t cap, int64_t* n_out);

/* Replace the per-point state (positions in the mesh's precision, point
 * classes 0 inner / 1 boundary, previous move distances as float64); host
 * pointers, any may be NULL to keep the current value.  Used to resume a
 * mesh or to start two implementations from identical states.  Positions are
 * checked on the device after the copy: a position that is not finite or lies
 * outside the SDF grid box returns TRIME_EINVAL (the message names the first
 * such point) and leaves the state unchanged. */
int mesh_set_state(mesh_t* m, const void* xy, const uint8_t* cls, const double* dprev);

/* The per-point state mesh_set_state replaces, in input order, into HOST
 * arrays of N_current entries (any may be NULL): positions in the mesh's
 * precision, classes (0 inner / 1 boundary), previous move distances as
 * float64.  Synchronous. */
int mesh_get_state(mesh_t* m, void* xy, uint8_t* cls, double* dprev);

/* Hybrid state: switched flag and the previous iteration's quality. */
int mesh_set_method_state(mesh_t* m, int32_t switched, double prev_half_alpha, double prev_half_beta,
                          double prev_max_alpha);

/* Per-point results of the last mesh_step iteration, in input order, float64:
 * what = 0 raw new position before treatment (2 per point), 1 DistMesh force F_i
 * (2), 2 CVD centroid (2), 3 sum of spring magnitudes |f| at the point (1),
 * 4 point class after treatment (1, as 0.0/1.0), 5 previous-move distance (1),
 * 6 quadrature level used (1).  Host buffer of cap doubles. */
int mesh_get_debug(mesh_t* m, int32_t what, double* out, int64_t cap);

/* Release all memory of m (NULL is ignored). */
void mesh_destroy(mesh_t* m);

/* Message of the last failure on the calling thread ("" if none). */
const char* mesh_last_error(void);

/* a1 on its own (Sec. 3.2 grid, App. B N_opt): counting sort of n points into
 * an nbx*nby bucket grid over [x0,x1]x[y0,y1].  All pointers are DEVICE
 * memory: x, y (n float64), out: bucket_start (nbx*nby+1 int32), sorted_idx
 * (n int32, input indices grouped by bucket, order within a bucket
 * unspecified).  scratch: device int32 array of at least 2*n + nbx*nby + 1024
 * entries, overwritten.  Asynchronous on the stream (cudaStream_t). */
int mesh_bucket_points(const double* x, const double* y, int64_t n, double x0, double y0, double x1,
                       double y1, int32_t nbx, int32_t nby, int32_t* bucket_start, int32_t* sorted_idx,
                       int32_t* scratch, void* cuda_stream);

/* Sec. 3.1: signed distance field of a closed loop of nv >= 3 line segments
 * given clockwise (HOST array xy of nv (x, y) float64 pairs; segment k runs
 * from vertex k to vertex k+1, the last back to vertex 0), sampled at the
 * nodes (x0 + i (x1-x0)/(nx-1), y0 + j (y1-y0)/(ny-1)) into out (nx*ny
 * float32, row-major out[j*nx + i], host or device memory), ready to pass as
 * a mesh_grid2d.  The value is the distance to the closest segment (FP64, the
 * smaller segment index on ties; closest point p* = a + t (b - a), t the
 * clamped projection), negative where (p - p*) . n > 0 with n the segment's
 * inward unit normal (right of its direction), or at an end point the sum of
 * the two incident segments' unit normals; rounded to float32.  The segments
 * are listed in a grid of cells about the mean segment length and searched
 * outwards as in Sec. 3.1, once per cell (the nodes of a cell then test only
 * its candidates).  Synchronous on cuda_stream; allocates and frees its
 * scratch.  Errors: TRIME_EINVAL (fewer than 3 vertices, a non-finite or
 * repeated vertex, a bad box or grid), TRIME_ECUDA. */
int mesh_segment_sdf_grid(const double* xy, int64_t nv, double x0, double y0, double x1, double y1, int32_t nx,
                          int32_t ny, float* out, void* cuda_stream);

/* Sec. 3.3 Eq. 7: the element sizing field mu(x) = min over the ns boundary
 * samples s (HOST array sxy of (x, y) float64 pairs) of K |s - x| + lfs(s)
 * (HOST array of ns local feature sizes, >= 0), K >= 0 the gradation, at the
 * nodes (x0 + i (x1-x0)/(nx-1), y0 + j (y1-y0)/(ny-1)) into out (nx*ny
 * float32, row-major, host or device memory), ready to pass as the sizing
 * mesh_grid2d.  Exact minimum in FP64 (the samples in a bucket grid, each
 * node searching outwards until no unvisited sample can do better), rounded
 * to float32.  Synchronous on cuda_stream.  Errors: TRIME_EINVAL, TRIME_ECUDA. */
int mesh_sizing_field(const double* sxy, const double* lfs, int64_t ns, double K, double x0, double y0, double x1,
                      double y1, int32_t nx, int32_t ny, float* out, void* cuda_stream);

/* Sec. 3.5: initial points for a mesh of n_init points (h_i and geps_i as
 * mesh_init would compute them for n_init points; p NULL = defaults, of
 * which eta, fac_geps, newton_max and damping are used).  The inner cells of
 * the SDF grid and the boundary cells whose midpoint SDF is at most
 * eta min(dx, dy) expect n^E = rho_norm n_init points (rho = 1/mu^2 at the
 * cell midpoint, normalised over those cells); in row-major order (rows
 * j = 0, 1, ...; i = 0, 1, ... within a row) each takes round(n^E + carried
 * residual) points (halves up, at least 0) and passes the residual in equal
 * parts to its selected neighbours not yet visited among (i+1, j), (i-1, j+1),
 * (i, j+1), (i+1, j+1) (Floyd-Steinberg).  The k-th point overall is uniform
 * in its cell: x = (x0 + i dx) + u dx, u = (h(2k) >> 11) 2^-53, y likewise
 * with h(2k+1), h(n) the SplitMix64 output of seed + (n+1) 0x9E3779B97F4A7C15;
 * a point of a boundary cell whose SDF exceeds the cell's geps is projected
 * by the damped Newton iteration of Sec. 4.3 and moved there when the result
 * is a boundary point (Sec. 4.3 classes; else it stays where it was drawn).
 * xy: HOST array of cap (x, y)
 * float64 pairs; *n_out = the number of points (which differs from n_init by
 * the residuals left at the last cells); TRIME_ECAPACITY if cap is smaller.
 * Synchronous. */
int mesh_init_points(const mesh_grid2d* sdf, const mesh_grid2d* sizing, int64_t n_init, uint64_t seed,
                     const mesh_params* p, double* xy, int64_t cap, int64_t* n_out, void* cuda_stream);

/* Sec. 3.3: medial-axis approximating points of the points of m (read as
 * boundary samples), from the triangles of its last triangulation (rebuilt
 * first if the points changed since): the Voronoi vertices of a cell are the
 * circumcentres of its triangles (create m with bounded = 0 and validity = 0
 * for the plain Delaunay triangles inside the SDF grid's box).  Per point,
 * in input order, v (HOST, 4 doubles) gets v1, the circumcentre farthest from
 * the point, and v2, the farthest one with (c - p) . (v1 - p) <= 0 (ties to
 * the smaller ascending vertex-index triple); flags (HOST, 1 byte) bit 0 /
 * bit 1 tell whether v1 / v2 exist.  Synchronous. */
int mesh_medial_points(mesh_t* m, double* v, uint8_t* flags);

/* The automatic sizing field of App. A and Sec. 3.3 for a clockwise loop of
 * nv >= 3 segments (HOST xy), on the node grid (x0 + i (x1-x0)/(nx-1),
 * y0 + j (y1-y0)/(ny-1)) whose cells serve as the geometry grid (dx, dy):
 *  1. boundary samples: every vertex, and floor(L/ds) evenly spaced points on
 *     each segment longer than ds = fac_s min(dx, dy) (fac_s 0.5), trimmed
 *     serially in index order (each unfinished point finds its closest other
 *     point whose midpoint with it has |sdf| <= fac_geps min(dx, dy), fac_geps
 *     0.01; if closer than ds that point is deleted and the current point
 *     moves to the midpoint, else the current point is finished; passes
 *     repeat until all are finished);
 *  2. their Delaunay triangles on the device (a mesh with bounded = 0 and
 *     validity = 0 on the segment SDF grid of mesh_segment_sdf_grid) and the
 *     medial points of mesh_medial_points (v1 then v2 of each sample);
 *  3. the medial points with at least n_thres = 3 others within
 *     r_nei = fac_nei n_thres ds (fac_nei 2) are kept (all if none would be);
 *     lfs of a sample is its distance to the closest kept one;
 *  4. mu on the grid by mesh_sizing_field with gradation K.
 * sdf_out (may be NULL) and sizing_out receive nx*ny float32 values (host or
 * device memory); counts (may be NULL) gets {samples, medial points, kept}.
 * Synchronous on cuda_stream.  Errors as the functions it uses. */
int mesh_auto_sizing(const double* xy, int64_t nv, double K, double x0, double y0, double x1, double y1,
                     int32_t nx, int32_t ny, float* sdf_out, float* sizing_out, int64_t* counts,
                     void* cuda_stream);

/* Exact signed distance (Sec. 3.1, the loop xy of nv clockwise vertices as
 * mesh_segment_sdf_grid, FP64, not rounded) at np points pts (x, y pairs),
 * by a search over every segment; pts and out in host or device memory.
 * Synchronous on cuda_stream.  Errors: TRIME_EINVAL, TRIME_ECUDA. */
int mesh_segment_sdf_points(const double* xy, int64_t nv, const double* pts, int64_t np, double* out,
                            void* cuda_stream);

/* Adaptive distance field (Sec. 3.7 and Fig. 17; App. B T_depth = 10,
 * fac_Etol = 0.1): one quadtree per listed cell of the node grid
 * (x0, y0, x1, y1, nx, ny; cell j (nx-1) + i spans nodes (i, j)..(i+1, j+1)).
 * A node's corners hold the exact signed distance to the clockwise loop xy
 * (mesh_segment_sdf_points); the bilinear values at its four edge midpoints
 * and its centre are compared with the exact distances there, and the node
 * splits into four children when the largest difference exceeds tol[r] of
 * its cell cells[r] and its level is below max_depth (0..14).  Node
 * coordinates: cell corner (x0 + i dx, y0 + j dy), node corner cx0 + ix
 * (dx 2^-L) at level L.  Nodes are numbered level by level, the four
 * children of a parent consecutive in the quadrant order (0,0), (1,0),
 * (0,1), (1,1) and in their parents' order.  cells (distinct) and tol
 * (finite, >= 0) are host arrays of ncells; the tree lives in device memory
 * until mesh_adf_destroy.  Synchronous on cuda_stream.  Errors: TRIME_EINVAL,
 * TRIME_ECAPACITY (more than 2^30 nodes), TRIME_ECUDA. */
typedef struct adf_s adf_t;
int mesh_adf_build(const double* xy, int64_t nv, double x0, double y0, double x1, double y1, int32_t nx, int32_t ny,
                   const int32_t* cells, const double* tol, int32_t ncells, int32_t max_depth, adf_t** out,
                   void* cuda_stream);

/* The boundary cells of m's geometry grid (Sec. 3.2 class 1), ascending, and
 * the tolerances E_tol,i = fac_etol geps_i sqrt(N_current / N_total)
 * (Sec. 3.7), into HOST arrays of cap entries; *n_out = the number of
 * boundary cells (TRIME_ECAPACITY if cap is smaller).  With mesh_adf_build
 * on m's SDF grid box and node counts this gives the paper's ADF of a mesh. */
int mesh_adf_cells(mesh_t* m, double fac_etol, int32_t* cells, double* tol, int64_t cap, int64_t* n_out);

/* Node and level counts of a. */
int mesh_adf_size(const adf_t* a, int64_t* n_nodes, int32_t* n_levels);

/* Node arrays into HOST buffers of cap nodes: v[4n] corners (v00, v10, v01,
 * v11), child[n] first child or -1, root[n] index into the cell list,
 * lev[3n] (level, ix, iy).  *n_out = the node count (TRIME_ECAPACITY if cap
 * is smaller). */
int mesh_adf_export(const adf_t* a, double* v, int32_t* child, int32_t* root, int32_t* lev, int64_t cap,
                    int64_t* n_out);

/* ADF values at np points pts (x, y pairs; host or device): the point's cell
 * by floor((x - x0) / dx), the leaf of its tree holding the point (a
 * coordinate equal to a midpoint goes to the upper child), bilinear in the
 * leaf; NaN where the cell has no tree.  out: np doubles, host or device.
 * Synchronous on cuda_stream. */
int mesh_adf_eval(const adf_t* a, const double* pts, int64_t np, double* out, void* cuda_stream);

/* Release the tree (NULL is ignored). */
void mesh_adf_destroy(adf_t* a);

/* mesh_bucket_points for callers that cannot allocate device memory: the
 * same counting sort (same arguments and outputs, all DEVICE pointers), but
 * its scratch is a fixed 16 MiB array inside the library instead of a
 * caller buffer, and it calls no cudaMalloc, cudaFree or allocating routine.
 * It serves callers whose device memory belongs to another allocator (a
 * framework pool that has reserved the GPU, where an extra cudaMalloc fails or
 * fragments it) and callers on latency-critical loops where cudaMalloc's
 * implicit synchronisation would stall other work.  Limit: 2*n + nbx*nby +
 * nbx*nby/4096 + 1 <= 4194304, else TRIME_EINVAL.  The first call on each
 * device resolves the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  All calls
 * on a device share the array and each call re-clears the part that must start
 * at zero: calls that overlap on the GPU (e.g. on two streams) race.  The paper
 * has no counterpart; asynchronous on the stream (cudaStream_t). */
int mesh_bucket_points_noalloc(const double* x, const double* y, int64_t n, double x0, double y0, double x1,
                               double y1, int32_t nbx, int32_t nby, int32_t* bucket_start, int32_t* sorted_idx,
                               void* cuda_stream);

/* Per-stage device timing (tracing): run n_iters iterations as separate
 * kernel launches (not the graph) with CUDA events between the stages on the
 * library's stream and ADD the elapsed milliseconds to stage_ms[0..6]:
 * 0 bucketing (a1), 1 Voronoi cells (a2), 2 triangle emission, validity and
 * quality sums (a3/a4/a8), 3 statistics and hybrid/termination decision,
 * 4 move and point treatment (a5-a7), 5 movement statistics, 6 whole
 * iteration.  Semantics otherwise as mesh_step.  Synchronises. */
int mesh_profile_step(mesh_t* m, int32_t n_iters, double* stage_ms);

/* Stop the iterations as soon as the minimum angle of a rebuild reaches
 * min_angle_deg (checked on the device after every rebuild).  While a target
 * is set it replaces the quality termination test of Sec. 4 (the relative
 * changes of the 1/2-means); the small-movement test stays.  0 removes the
 * target.  Setting a target the mesh has not reached clears a previous
 * termination.  Used to measure the wall time to a given quality.
 * Synchronises. */
int mesh_set_quality_target(mesh_t* m, double min_angle_deg);

/* Tiling of the iteration: size the bucket grid for n_opt points per bucket
 * (> 0; the default is mesh_params.N_opt) and clip each Voronoi cell with
 * `lanes` = 8 (four cells per warp; cells needing more than 8 edges at some
 * step redone with 16, and from there with 32 lanes), 16 (two cells per warp,
 * then 32) or 32 lanes (one cell per warp); the default is 8.  The results do
 * not depend on either choice, only the speed does.  Re-captures the iteration graph;
 * synchronises.  Errors: TRIME_EINVAL, TRIME_ENOMEM, TRIME_ECUDA. */
int mesh_set_tuning(mesh_t* m, double n_opt, int32_t lanes);

/* Verification hook for the exact predicates the Voronoi kernel uses
 * (Sec. 2.1 cell cutting decisions): for each of nq queries of four points
 * a, b, c, d (HOST array pts of nq*8 doubles, x/y interleaved) and their ids
 * (HOST nq*4 int32), evaluates on the device out_orient[q] = sign of
 * orient2d(a, b, c) and out_incircle[q] = sign of the symbolically perturbed
 * det of rows [x, y, x^2+y^2, 1] (> 0 iff d is inside circle(a, b, c) for
 * counter-clockwise a, b, c; ties broken by perturbing the lift of point r by
 * eps^(id_r + 1)).  A value of 2 reports the capacity/underflow guard.
 * Synchronous; host output arrays of nq int32 each. */
int mesh_exact_predicates(const double* pts, const int32_t* ids, int64_t nq, int32_t* out_orient,
                          int32_t* out_incircle);

/* Verification hook of the tensor-core tile used by the learned model:
 * D = A * B^T with A (M x K) and B (N x K) given as BF16 bit patterns
 * (row-major HOST arrays of uint16) and D (M x N) a row-major HOST float32
 * array, multiplied by tcgen05 MMAs on the device with FP32 accumulation in
 * tensor memory.  M a positive multiple of 128; N and K multiples of 16 in
 * [16, 256].  Synchronous.  TRIME_ETIMEOUT if a bounded device wait ran out.
 * The paper has no counterpart (its method has no learned part). */
int mesh_tc_gemm_bf16(const uint16_t* A, const uint16_t* B, float* D, int32_t M, int32_t N, int32_t K);

/* ---------------------------------------------------------------- learned proposals
 * A small network proposes, for every point, its displacement over the next
 * iterations of the plain method; plain iterations remain the fallback and
 * judge every proposal by the quality they measure (Sec. 3.6 Eqs. 11-12 and
 * the minimum angle).  The paper's method has no learned part; this is an
 * addition of this library.
 *
 * Network: 48 BF16 inputs (39 features, zero-padded), two hidden layers of
 * 64 ReLU units, 2 outputs (the proposed displacement divided by h_i);
 * BF16 weights and activations, FP32 accumulation, all products on the
 * tensor cores.  Parameters: a flat FP32 vector of TRIME_MLP_PARAMS values,
 * W1 (64 x 48, row-major), b1 (64), W2 (64 x 64), b2 (64), W3 (2 x 64), b3 (2).
 * Features of point i, in order: the offsets (x_j - x_i, y_j - y_i) r_i of
 * its 16 nearest other points (by squared distance, ties by smaller index,
 * nearest first), r_i = 1 / h_i rounded once to FP64; ln(h_i / h_avg)
 * (Sec. 3.7); the gradient of the sizing field at p_i; 1 if p_i is a boundary
 * point (Sec. 4.3); 1 if the next move is CVD; the point's last move times
 * r_i (zero when unknown: the positions
 * before the last iteration are recorded by mesh_step_learned and
 * mesh_collect_pairs, not by mesh_step); each rounded to float32 and then to
 * BF16 (nearest, ties to even). */
#define TRIME_MLP_IN 48
#define TRIME_MLP_PARAMS 7426
typedef struct mlp_s mlp_t;

/* Create a model on the current device: parameters from a HOST array of
 * TRIME_MLP_PARAMS floats, or (params == NULL) a seeded He initialisation
 * with zero biases.  Work is ordered on cuda_stream.  Errors: TRIME_EINVAL
 * (non-finite parameter), TRIME_ENOMEM, TRIME_ECUDA. */
int mlp_create(mlp_t** out, const float* params, uint64_t seed, void* cuda_stream);
void mlp_destroy(mlp_t* m);
/* Copy the FP32 parameters to / from a HOST array of TRIME_MLP_PARAMS floats;
 * setting them also resets the optimiser state. */
int mlp_get_params(mlp_t* m, float* params);
int mlp_set_params(mlp_t* m, const float* params);
/* Y (n x 2 float32) = network(X) for X (n x 48 BF16 bit patterns), both host
 * or both device arrays (detected).  Synchronous. */
int mlp_forward(mlp_t* m, const uint16_t* X, int64_t n, float* Y);
/* Loss L = sum over the n samples and 2 outputs of (Y - T)^2 / (2n) and its
 * gradient with respect to the parameters (HOST array of TRIME_MLP_PARAMS
 * floats, same layout), computed by the device's forward and backward
 * kernels.  X, T host or device.  Synchronous. */
int mlp_loss_grad(mlp_t* m, const uint16_t* X, const float* T, int64_t n, double* loss, float* grad);
/* Adam (beta 0.9 / 0.999, eps 1e-8, step lr) over `epochs` shuffled passes of
 * mini-batches of `batch` (>= 128) samples of the DEVICE arrays X (n x 48
 * BF16) and T (n x 2 float32); *last_loss (may be NULL) = mean batch loss of
 * the last epoch.  Synchronous. */
int mlp_train(mlp_t* m, const uint16_t* X, const float* T, int64_t n, int32_t epochs, int32_t batch, double lr,
              uint64_t seed, double* last_loss);

/* Features of every point of m at its current positions, in input order:
 * X (n x 48 BF16 bits) and, if h is not NULL, h_i (n float32); host or
 * device arrays.  Synchronous. */
int mesh_features(mesh_t* m, uint16_t* X, float* h);

/* Training pairs from m's own trajectory: one plain iteration, then the
 * features (with that iteration's move) into X (DEVICE, n x 48 BF16) and,
 * after `horizon` more plain iterations, the displacement of every point over
 * them divided by its h_i into T (DEVICE, n x 2 float32), input order.
 * Advances m by horizon + 1 iterations.  Synchronous. */
int mesh_collect_pairs(mesh_t* m, int32_t horizon, uint16_t* X, float* T);

/* Move every point to p_i + h_i * network(features_i), the move clamped to
 * jump * fac_pt * h_i and treated as in Sec. 4.3 (no rebuild, no quality
 * check).  Synchronous. */
int mesh_propose(mesh_t* m, mlp_t* net, double jump);

/* mesh_step with a proposal before every `every`-th iteration (every >= 1):
 * from the same state, one plain iteration and the proposal followed by one
 * plain iteration both run; the proposal branch is kept if its quality beats
 * the plain branch's (1/2-mean of alpha smaller, minimum angle not smaller by
 * more than min_angle_tol degrees, no capacity guard tripped), otherwise the
 * plain branch's state is restored.  Both branches count as iterations.  At most max_proposals proposals are made (<= 0: no limit);
 * the iterations after the last one are plain.  *accepted / *rejected (may be
 * NULL) count the proposals.  Statistics and termination as mesh_step (stats
 * may not be NULL).  TRIME_EINVAL while N_current < N_total (point
 * addition); mesh_features, mesh_collect_pairs and mesh_propose likewise. */
int mesh_step_learned(mesh_t* m, mlp_t* net, int32_t n_iters, int32_t every, double jump, double min_angle_tol,
                      int32_t max_proposals, mesh_stats* stats, int32_t* accepted, int32_t* rejected);

/* Measured issue peaks of the FP32 and FP64 pipes of the current device
 * (TFLOP/s; 8 independent fused multiply-add chains per thread, 8 blocks of
 * 256 threads per SM), with the SM count and the nominal SM clock (kHz) the
 * device reports: the roofline denominators of the arithmetic-bound kernels.
 * sm_count and sm_clock_khz may be NULL.  Synchronous; about 0.1 s.  The paper
 * has no counterpart. */
int mesh_measure_pipe_peaks(double* fp32_tflops, double* fp64_tflops, int32_t* sm_count, int32_t* sm_clock_khz);

/* ---------------------------------------------------------------- batches
 * Many independent meshes of uneven sizes stepped together: every stage of
 * an iteration is one kernel launch over all meshes (their points are
 * concatenated on the device, each mesh padded to a multiple of 256 slots so
 * a thread block or warp never mixes meshes), and one CUDA graph replays the
 * whole batch's iteration.  Each mesh keeps its own grids, geometry grid,
 * bucket grid, fac_mu, quality statistics, hybrid switch and termination
 * (Sec. 2.4, 4.2, 4); a mesh that has terminated is skipped by every kernel
 * while the others continue.  Per mesh, the results are those of a mesh_t
 * created with the same inputs (triangles identical, moves equal up to the
 * order of floating-point sums).  The paper treats one mesh at a time; the
 * batch is this library's production form for many small meshes. */
typedef struct mesh_batch_s mesh_batch_t;

/* What mesh_batch_init's autotuner chose and what it measured. */
typedef struct {
    double n_opt;             /* points per bucket the bucket grids are sized for     */
    int32_t lanes;            /* Voronoi lanes per cell of the first pass: 8, 16 or 32 */
    int32_t n_candidates;     /* candidates timed (0 without autotuning)              */
    int64_t n_slots;          /* device slots: the meshes' points plus padding        */
    int64_t n_buckets;        /* buckets of all meshes, one pad bucket per mesh added */
    double cand_n_opt[12];
    int32_t cand_lanes[12];
    double cand_ms[12];       /* device time of one rebuild (a1..a4) per candidate    */
} mesh_tuning;

/* Create a batch of n_meshes (1 .. 2^20) meshes on the current device.
 *  sdfs, sizings: n_meshes host grids each (as mesh_init); xys: n_meshes
 *  HOST point arrays (precision as p->precision); ns: n_meshes point counts
 *  (>= 0; total padded size <= 2^30).  One parameter set p (NULL: defaults)
 *  serves every mesh.  autotune != 0: time one rebuild per candidate of
 *  (points per bucket in {2/3, 1, 3/2} x p->N_opt) x (8, 16 or 32 Voronoi
 *  lanes per cell) on these inputs and keep the fastest (the triangles do not
 *  depend on the choice); autotune == 0 uses p->N_opt and 8 lanes.  Errors as
 *  mesh_init; a message names the offending mesh.  Point addition is not
 *  available in a batch (p->n_total above a mesh's n: TRIME_EINVAL). */
int mesh_batch_init(mesh_batch_t** out, int32_t n_meshes, const mesh_grid2d* sdfs, const mesh_grid2d* sizings,
                    const void* const* xys, const int64_t* ns, const mesh_params* p, int32_t autotune,
                    void* cuda_stream);

/* Number of meshes (0 for NULL). */
int mesh_batch_size(const mesh_batch_t* b);

/* mesh_rebuild for every mesh; stats: NULL or n_meshes entries. */
int mesh_batch_rebuild(mesh_batch_t* b, mesh_stats* stats);

/* Up to n_iters iterations of every mesh that has not terminated (one graph
 * launch each); stops early once every mesh has terminated.  stats: NULL
 * (asynchronous) or n_meshes entries, each with that mesh's iteration count. */
int mesh_batch_step(mesh_batch_t* b, int32_t n_iters, mesh_stats* stats);

/* mesh_get_triangles / mesh_get_points / mesh_set_state /
 * mesh_set_method_state for mesh index `mesh` of the batch (0-based, point
 * indices local to that mesh). */
int mesh_batch_get_triangles(mesh_batch_t* b, int32_t mesh, int32_t* tri, int64_t cap, int64_t* n_out);

/* mesh_quality for one mesh of the batch. */
int mesh_batch_quality(mesh_batch_t* b, int32_t mesh, mesh_quality_stats* q);
int mesh_batch_get_points(mesh_batch_t* b, int32_t mesh, void* xy, int64_t cap, int64_t* n_out);
int mesh_batch_set_state(mesh_batch_t* b, int32_t mesh, const void* xy, const uint8_t* cls, const double* dprev);
int mesh_batch_set_method_state(mesh_batch_t* b, int32_t mesh, int32_t switched, double prev_half_alpha,
                                double prev_half_beta, double prev_max_alpha);

/* mesh_profile_step for the whole batch. */
int mesh_batch_profile_step(mesh_batch_t* b, int32_t n_iters, double* stage_ms);

/* mesh_set_quality_target for one mesh of the batch, or all of them (mesh = -1). */
int mesh_batch_set_quality_target(mesh_batch_t* b, int32_t mesh, double min_angle_deg);

/* mesh_set_tuning for the whole batch (e.g. to reuse an earlier autotuning
 * result without timing again). */
int mesh_batch_set_tuning(mesh_batch_t* b, double n_opt, int32_t lanes);

/* mesh_step_learned for every mesh of the batch at once (the batched form
 * with the learned part; the paper has no learned part).  Before every
 * `every`-th iteration all meshes that have not terminated get a proposal
 * round: from the same state one plain iteration and the proposal followed by
 * one plain iteration run for the whole batch, then each mesh keeps the
 * branch its own statistics favour (the rule of mesh_step_learned) and the
 * meshes whose proposal lost are restored to their plain branch.  At most
 * max_rounds rounds (<= 0: no limit).  stats (not NULL), accepted and
 * rejected (may be NULL): n_meshes entries each, per mesh.  The features'
 * "move in use" is each mesh's own (CVD once its hybrid has switched).
 * Synchronous.  Errors as mesh_batch_step; TRIME_ETIMEOUT if a tensor-core
 * wait of the model ran out. */
int mesh_batch_step_learned(mesh_batch_t* b, mlp_t* net, int32_t n_iters, int32_t every, double jump,
                            double min_angle_tol, int32_t max_rounds, mesh_stats* stats, int32_t* accepted,
                            int32_t* rejected);

/* The autotuner's choice and timings. */
int mesh_batch_get_tuning(const mesh_batch_t* b, mesh_tuning* out);

/* Release all memory of b (NULL is ignored). */
void mesh_batch_destroy(mesh_batch_t* b);

#ifdef __cplusplus
}
#endif
#endif
