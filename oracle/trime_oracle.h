/*
 * trime_oracle.h -- plain FP64 CPU oracle for one TriMe++ meshing iteration.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py may load this code.  The product
 * path (the CUDA library under paper_2309_13824_gb300/) shares no code with it.
 *
 * What it computes, with the paper section each part follows
 * (TriMe++, Lu & Rycroft, arXiv 2309.13824):
 *   - geometry grid classes, h_i, geps_i                      Sec. 3.2, 3.4, 3.7
 *   - bounded Voronoi cells by half-plane clipping            Sec. 2.1 Fig. 3, Sec. 4.1
 *   - Delaunay triangles read off the cells, Tests 1-3        Sec. 4.1, Procedure I
 *   - DistMesh spring forces + forward Euler                  Sec. 2.2 Eqs. 2-5
 *   - CVD density-weighted centroid, adaptive quadrature      Sec. 2.3 Eq. 6, Sec. 4.2
 *   - point treatment: clamp, classify, sphere trace, Newton  Sec. 4.3 Eqs. 8-10
 *   - aspect/edge ratio quality, 1/2-means, hybrid switch     Sec. 3.6 Eqs. 11-12, Sec. 4
 *   - point addition at the centroids of the triangles with   Sec. 3.6, Sec. 3.7
 *     the largest R_circ / h_i, quantities rescaled
 *   - signed distance from clockwise line segments            Sec. 3.1
 *   - element sizing field from boundary samples and lfs      Sec. 3.3 Eq. 7
 *   - boundary samples, medial axis, local feature size       App. A, Sec. 3.3
 *   - point initialisation with Floyd-Steinberg dithering      Sec. 3.5
 *   - adaptive distance field (quadtrees on boundary cells)    Sec. 3.7 (Fig. 17), App. B
 *
 * Every sign decision of the triangulation (incircle / orientation) is exact:
 * big-integer arithmetic behind a deliberately loose double-precision filter,
 * with symbolic perturbation of the lifted coordinate for exact ties.
 */
#ifndef TRIME_ORACLE_H
#define TRIME_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t nx, ny;            /* nodes, >= 2 each                      */
    double x0, y0, x1, y1;     /* node (0,0) at (x0,y0), (nx-1,ny-1) at (x1,y1) */
    const float* v;            /* row-major v[j*nx+i], borrowed          */
} om_grid;

typedef struct {
    int32_t method;            /* 0 DistMesh, 1 CVD, 2 hybrid            */
    int32_t bounded;           /* 1: octagon bound of span S (Sec. 4.1); 0: domain box only */
    int32_t validity;          /* 1: Tests 1-3 (Sec. 4.1); 0: keep every emitted triangle */
    int32_t newton_max;        /* T_ct^newton = 10                       */
    int32_t trace_max;         /* sphere-trace step cap (paper silent)   */
    int32_t quad_max_level;    /* quadrature level cap (paper silent)    */
    double fac_F, k_spring, dt;
    double fac_pt, fac_geps, fac_voro_bound, fac_end;
    double T_circ, T_switch, T_end_q, T_end_amax;
    double N_opt, eta, damping;
    double fac_retria;         /* DistMesh re-triangulation threshold factor (Algorithm 1, App. B: 0.1); 0: every iteration */
    double fac_add;            /* point addition: N_add = min(floor(fac_add N_current), N_total - N_current) (Sec. 3.6, App. B: 0.6) */
    double T_add;              /* point addition quality threshold T_quality^add (Sec. 3.6, App. B: 0.002) */
    int64_t n_total;           /* N_total; above the initial n it runs the point-addition scheme (Sec. 3.6) */
} om_params;

typedef struct {
    int64_t n_tri;             /* valid triangles                        */
    int64_t n_edges;           /* unique valid edges                     */
    double half_mean_alpha;    /* M_1/2(alpha), Eq. 12                   */
    double half_mean_beta;     /* M_1/2(beta)                            */
    double max_alpha, max_beta, min_angle_deg;
    double mean_size_dev;      /* mean |l/(fac_mu mu(m)) - 1| over valid edges */
    double fac_mu;             /* Eq. 3                                  */
    int64_t newton_fail, trace_cap, quad_cap, clip_errors;
    int32_t method_used;       /* 0 DM / 1 CVD for the move just made    */
    int32_t terminated;        /* termination test held (Sec. 4)         */
    int32_t switched;          /* hybrid has switched to CVD             */
    int32_t small_moves;       /* all inner moves < fac_end h_i          */
    int32_t triangulated;      /* the step re-triangulated (Algorithm 1)  */
    int64_t added;             /* points the step added (Sec. 3.6)        */
    int64_t n_points;          /* N_current after the step                */
} om_stats;

typedef struct om_mesh om_mesh;

void om_default_params(om_params* p);

/* Create from positions xy[2n] (x,y interleaved).  Grids are deep-copied.
 * With p->n_total > n the mesh starts with N_current = n points and grows to
 * N_total by the point-addition scheme (Sec. 3.6); h_i is computed from
 * N_current (Sec. 3.7).  Returns NULL on invalid input (message via
 * om_last_error). */
om_mesh* om_create(const om_grid* sdf, const om_grid* sizing, const double* xy,
                   int64_t n, const om_params* p);
void om_destroy(om_mesh* m);
const char* om_last_error(void);

/* Procedure I at the current positions: cells, triangles, validity, quality. */
int om_rebuild(om_mesh* m);
/* One meshing iteration: rebuild, quality, hybrid/termination logic, move.
 * While N_current < N_total the termination tests and the hybrid switch are
 * not evaluated; an iteration whose 1/2-means of alpha and beta both changed
 * by less than T_add instead adds points (no move in that iteration). */
int om_step(om_mesh* m);
/* Same as om_step but only for the cells listed (timing sample; no move). */
int om_rebuild_sample(om_mesh* m, const int64_t* cells, int64_t ncells, int with_centroid);
/* The valid triangles owned by the given cells (Procedure I restricted to
 * them; a triangle is owned by its smallest-index vertex), as index triples
 * (smallest first, counter-clockwise) into tri (capacity cap triples).
 * Returns the number of such triangles (may exceed cap; then only cap are
 * written). */
int64_t om_sample_triangles(om_mesh* m, const int64_t* cells, int64_t ncells, int32_t* tri, int64_t cap);

/* om_rebuild_sample's work spread over nthreads OpenMP threads (timing only);
 * returns the number of owned valid triangles of the cells. */
int64_t om_rebuild_sample_mt(om_mesh* m, const int64_t* cells, int64_t ncells, int with_centroid, int nthreads);

int64_t om_num_points(const om_mesh* m);
/* OpenMP threads of the per-cell loops of om_rebuild / om_step (cells,
 * emission, centroids, point treatment); 1 (the default) runs serially.
 * Results do not depend on it. */
void om_set_threads(om_mesh* m, int threads);
int64_t om_num_triangles(const om_mesh* m);
void om_get_triangles(const om_mesh* m, int32_t* tri);          /* 3*n_tri, sorted */
int64_t om_num_edges(const om_mesh* m);
void om_get_edges(const om_mesh* m, int32_t* e);                /* 2*n_edges, sorted */
void om_get_points(const om_mesh* m, double* xy);
void om_set_points(om_mesh* m, const double* xy);
void om_get_class(const om_mesh* m, uint8_t* cls);
void om_set_class(om_mesh* m, const uint8_t* cls);
void om_get_dprev(const om_mesh* m, double* d);
void om_set_dprev(om_mesh* m, const double* d);
void om_set_method_state(om_mesh* m, int32_t switched, double prev_a, double prev_b, double prev_amax);
/* Results of the last om_step: raw move p_new before treatment, force F (DM)
 * or centroid c (CVD), and the quadrature level used per point. */
void om_get_pnew(const om_mesh* m, double* xy);
void om_get_force(const om_mesh* m, double* f);
void om_get_fsum(const om_mesh* m, double* s);   /* sum_e |f_e| per point (force scale) */
void om_get_centroid(const om_mesh* m, double* c);
void om_get_cell_area(const om_mesh* m, double* a);
void om_get_quad_level(const om_mesh* m, int32_t* lv);
void om_get_stats(const om_mesh* m, om_stats* s);

/* The mesh-quality statistics the paper tabulates at termination (Sec. 5:
 * median, mean, maximum, standard deviation of alpha and beta, shares with
 * alpha < 1.2 and < 2) of the valid triangles of the last rebuild, at the
 * current positions (call after om_rebuild), plus the minimum angle, the
 * alpha histogram (bin k: [e_k, e_{k+1}), e = 1, 1.05, 1.1, 1.2, 1.3, 1.5,
 * 2, 3, 5, 10, inf; values below 1 in bin 0) and |l / (fac_mu mu(m)) - 1|
 * over the valid edges by mean and 95th percentile.  Medians: the value of
 * rank floor((n-1)/2) of the sorted values; the percentile: rank
 * ceil(0.95 n) - 1 (nearest rank). */
typedef struct {
    int64_t n_tri, n_edges;
    double median_alpha, median_beta, mean_alpha, mean_beta, max_alpha, max_beta, std_alpha, std_beta;
    double frac_alpha_lt_1_2, frac_alpha_lt_2, min_angle_deg;
    int64_t alpha_hist[10];
    double fac_mu, mean_size_dev, p95_size_dev;
} om_quality;
void om_quality_report(const om_mesh* m, om_quality* q);

/* Per-cell views for pins. */
int om_get_ring(const om_mesh* m, int64_t i, int32_t* labels, int cap);
int om_get_cell_polygon(const om_mesh* m, int64_t i, double* xy, int cap);
void om_get_geometry(const om_mesh* m, uint8_t* cls, double* h, double* geps, double* havg);
int om_point_cell(const om_mesh* m, double x, double y, int32_t* gi, int32_t* gj);

/* Exact predicates (sign in {-1,0,1}); incircle is det of rows
 * [x, y, x^2+y^2, 1] of (a,b,c,d): > 0 iff d is inside circle(a,b,c) for
 * counter-clockwise a,b,c.  The _sos form never returns 0. */
int om_orient2d(const double* a, const double* b, const double* c);
int om_incircle(const double* a, const double* b, const double* c, const double* d);
int om_incircle_sos(const double* a, int64_t ia, const double* b, int64_t ib,
                    const double* c, int64_t ic, const double* d, int64_t id);
double om_bilinear(const om_grid* g, double x, double y);

/* Sec. 3.1 signed distance from a closed loop of line segments given
 * clockwise (vertex k to k+1, the last back to the first; nv >= 3), at np
 * points (px, py): the distance to the closest segment (FP64, the smaller
 * segment index on ties; closest point p* = a + t (b - a), t the clamped
 * projection), negative where (p - p*) . n > 0 with n the segment's inward
 * unit normal (right of its direction), or at an end point the sum of the
 * two incident segments' unit normals; positive elsewhere.  Brute force over
 * all segments.  Returns 0, or -1 on bad input. */
int om_segment_sdf(const double* xy, int64_t nv, const double* px, const double* py, int64_t np, double* out);

/* Sec. 3.7: adaptive distance field.  One quadtree per listed grid cell
 * cells[r] = j (nx - 1) + i of the node grid (x0, y0, x1, y1, nx, ny), built
 * top-down: a node's four corners hold the exact segment SDF (om_segment_sdf);
 * the bilinear values at its four edge midpoints and its centre are compared
 * with the exact SDF there, and the node splits into four children when the
 * largest error exceeds tol[r] and its level is below max_depth.  Nodes are
 * numbered level by level, children in their parent's order, each parent's
 * four children consecutive in the quadrant order (0,0), (1,0), (0,1),
 * (1,1).  Coordinates: cell corner cx0 = x0 + i dx, node corner
 * cx0 + ix (dx 2^-L), the midpoints at level L + 1.  Returns a handle, or
 * NULL on bad input. */
typedef struct om_adf om_adf;
om_adf* om_adf_build(const double* xy, int64_t nv, double x0, double y0, double x1, double y1, int32_t nx, int32_t ny,
                     const int32_t* cells, const double* tol, int32_t ncells, int32_t max_depth);
int64_t om_adf_size(const om_adf* a);
/* Node arrays: v[4n] corners (v00, v10, v01, v11), child[n] first child or
 * -1, root[n] index into cells, lev[3n] (level, ix, iy). */
void om_adf_export(const om_adf* a, double* v, int32_t* child, int32_t* root, int32_t* lev);
/* ADF values at np points: the leaf of the point's cell tree holding it
 * (a coordinate equal to a midpoint goes to the upper child), bilinear in the
 * leaf; NaN where the point's cell has no tree. */
void om_adf_eval(const om_adf* a, const double* px, const double* py, int64_t np, double* out);
void om_adf_free(om_adf* a);

/* Eq. 7 element sizing field mu(x) = min over the boundary samples s of
 * K |s - x| + lfs(s) (Sec. 3.3), at np points; brute force over the ns
 * samples sxy (x, y pairs) with local feature sizes lfs.  Returns 0, or -1
 * on bad input. */
int om_sizing_field(const double* sxy, const double* lfs, int64_t ns, double K, const double* px, const double* py,
                    int64_t np, double* out);

/* App. A: boundary samples of a clockwise segment loop: every vertex and,
 * on each segment longer than ds, floor(L/ds) evenly spaced interior points
 * (spacing below ds), in segment order; then the serial trimming: in index
 * order, each unfinished point finds its closest other point whose midpoint
 * m with it has |sdf(m)| <= geps_hat (Sec. 3.1 segment SDF; ties by index);
 * if that point is closer than ds it is deleted and the current point moves
 * to m, otherwise the current point is finished; passes repeat until every
 * point is finished.  Writes up to cap (x, y) pairs; returns the count or -1. */
int64_t om_boundary_samples(const double* xy, int64_t nv, double ds, double geps_hat, double* out, int64_t cap);

/* Sec. 3.3: medial-axis points of the points of m (boundary samples), read
 * off the Delaunay triangles of the last om_rebuild (Voronoi vertices =
 * circumcentres, fixed formula on the canonical order): v1 the circumcentre
 * of an incident triangle farthest from the point, v2 the farthest one with
 * (c - p) . (v1 - p) <= 0; ties to the smaller vertex-index triple.  v gets
 * 4 doubles per point (v1, v2), flags bit 0 = v1 exists, bit 1 = v2 exists. */
void om_medial_points(const om_mesh* m, double* v, uint8_t* flags);

/* Sec. 3.3: the medial points (nm (x, y) pairs) with at least n_thres others
 * within r_nei are kept (all of them if none would be); lfs of each sample =
 * its distance to the closest kept point.  Returns the number kept or -1. */
int64_t om_lfs(const double* sxy, int64_t ns, const double* mxy, int64_t nm, double r_nei, int32_t n_thres,
               double* lfs);

/* Sec. 3.5 point initialisation: the inner and selected boundary cells of the
 * geometry grid (the SDF grid's cells; a boundary cell is selected when the
 * SDF at its midpoint is at most eta min(dx, dy)) expect n^E = rho_norm n_init
 * points (rho = 1/mu^2 at the midpoint, normalised over the selected cells).
 * In row-major order (rows j = 0, 1, ..., columns i = 0, 1, ... within a row)
 * each selected cell takes round(n^E + carried residual) points (at least 0;
 * halves round up) and passes the residual in equal parts to its selected
 * neighbours not yet visited among (i+1, j), (i-1, j+1), (i, j+1), (i+1, j+1).
 * The k-th point overall is uniform in its cell: x = (x0 + i dx) + u dx with
 * u = (h(2k) >> 11) 2^-53, y likewise with h(2k+1), where h(n) is the
 * SplitMix64 output of seed + (n+1) 0x9E3779B97F4A7C15.  A point of a
 * selected boundary cell whose SDF exceeds that cell's geps is projected by
 * the damped Newton step of Sec. 4.3 (h_i and geps_i from N = n_init); the
 * projection counts when it ends as a boundary point (Sec. 4.3 classes),
 * otherwise the point stays where it was drawn.  Writes
 * up to cap (x, y) pairs in that order; returns the count, or -1. */
int64_t om_init_points(const om_grid* sdf, const om_grid* sizing, int64_t n_init, uint64_t seed, const om_params* p,
                       double* out, int64_t cap);
uint64_t om_splitmix64(uint64_t seed, uint64_t n);

/* Standalone pieces for pins. */
int om_polygon_centroid(const om_grid* sizing, const double* gen, const double* poly, int nv,
                        double eps_c, int max_level, double* c, int32_t* level);
int om_project_point(om_mesh* m, const double* p_old, int old_class, const double* p_new,
                     double* p_final, int32_t* new_class);

#ifdef __cplusplus
}
#endif
#endif
