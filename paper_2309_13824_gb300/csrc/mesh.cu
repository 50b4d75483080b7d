// mesh.cu -- host runtime behind the C ABI of include/trime.h.
//
// Owns every device buffer, precomputes the geometry grid once (TriMe++
// Sec. 3.2 cell classes, Sec. 3.4-3.5 density, Sec. 3.7 h_i and geps_i) with
// serial row-major sums, and captures one meshing iteration (a1..a8) into a
// CUDA graph that mesh_step replays.  Work runs on a private stream that is
// ordered after / before the caller's stream with events, so graph capture
// works whatever stream the caller passes.
//
// A mesh_t holds one mesh; a mesh_batch_t holds several independent meshes
// whose slots are concatenated (each padded to whole chunks of kChunk slots)
// and stepped by the same launches: one launch per stage covers every mesh,
// each block or warp reading its mesh's view from a device table.  The
// batch's bucket size and Voronoi lane count can be picked by timing the
// candidates on the batch itself (autotuning at mesh_batch_init).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "trime.h"

using namespace trime;

static thread_local std::string g_err;

static int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

namespace trime {
int set_error(int code, const char* msg) { return fail(code, msg); }
}  // namespace trime

#define CUDA_TRY(x)                                                                            \
    do {                                                                                       \
        cudaError_t e_ = (x);                                                                  \
        if (e_ != cudaSuccess) return fail(TRIME_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// one mesh of a mesh_s
struct Part {
    int64_t n = 0;
    int32_t soff = 0, npad = 0;  // first slot, padding slots after the points
    int32_t boff = 0, nb = 0;    // first bucket, buckets
    int32_t c0 = 0, c1 = 0;      // chunks (blocks of the emit / update kernels)
    DevParams dp{};
    DevGrid sdf{}, siz{};
    uint8_t* gcls = nullptr;
    double* gh = nullptr;
    double* ggeps = nullptr;
    uint8_t* gidist = nullptr;
    double rho_eff = 0;          // point-weighted mean point density
};

struct TuneCand {
    double nopt;
    int lanes;
    double ms;
};

struct LearnBufs;

struct mesh_s {
    int prec = 0;
    bool batched = false;
    int64_t nslots = 0;          // slots of all parts
    mesh_params P{};
    std::vector<Part> parts;
    int nbtot = 0;               // buckets in use (pad buckets included)
    int nbcap = 0;               // buckets allocated
    int lanes = 8;               // Voronoi lanes per cell of the first pass
    double nopt = 3.3;           // points per bucket the grids are sized for
    std::vector<TuneCand> tune;  // autotuning record
    struct QualityScratch* qs = nullptr;
    cudaStream_t user = nullptr, st = nullptr;
    cudaEvent_t ev = nullptr;
    void *cx = nullptr, *cy = nullptr, *cdp = nullptr, *sx = nullptr, *sy = nullptr, *sdp = nullptr;
    void *wx = nullptr, *wy = nullptr, *wdp = nullptr;  // DistMesh iterations that keep the triangulation
    uint8_t* wcls = nullptr;
    bool tri_stale = false;  // the sorted order no longer matches the triangulation
    int32_t *cid = nullptr, *sid = nullptr;
    uint8_t *ccls = nullptr, *scls = nullptr;
    int32_t *cell = nullptr, *key = nullptr, *rank = nullptr, *skey = nullptr, *sidx = nullptr;
    uint8_t* dom = nullptr;
    int32_t *bcount = nullptr, *bstart = nullptr, *scan_tmp = nullptr;
    int32_t* ring = nullptr;
    uint8_t* ring_n = nullptr;
    int32_t *warm = nullptr, *perm = nullptr;
    float* cellR = nullptr;
    uint64_t* vmask = nullptr;
    EmitPartial* ep = nullptr;
    UpdatePartial* up = nullptr;
    int nblk = 1;
    DevCtrl* ctrl = nullptr;     // [parts]
    DevCtrl* hctrl = nullptr;    // pinned host copy [parts]
    int32_t* ovf_n = nullptr;
    MeshView* dviews = nullptr;  // [parts] (batch)
    int32_t* cmesh = nullptr;    // [nslots / kChunk] (batch)
    double* dbg = nullptr;
    int32_t *tcnt = nullptr, *toff = nullptr, *tbuf = nullptr;
    int32_t* ovf_list = nullptr;
    float4* pf = nullptr;
    float2* pf3 = nullptr;
    float* pS = nullptr;
    void* xybuf = nullptr;
    cudaGraphExec_t gexec = nullptr;
    LearnBufs* learn = nullptr;
    // point addition (single mesh): capacity N_total and the selection scratch
    int64_t ncap = 0;
    int64_t added_call = 0;      // points added during the current mesh_step
    void* akeys = nullptr;       // [2 ncap + 16] selection keys
    int32_t *ahist = nullptr, *hhist = nullptr;  // 256 device / pinned host
    int32_t *acnt = nullptr, *aoff = nullptr;    // [ncap + 1] per-owner counts and offsets by id
    int32_t *chk = nullptr, *hchk = nullptr;     // state-check result: device / pinned host
    std::vector<void*> allocs;
};

struct mesh_batch_s : mesh_s {};

// scratch of the quality report, allocated on its first use
struct QualityScratch {
    QBufs b{};
    int64_t cap_t = 0, cap_e = 0;
};

// learned proposals: scratch and the saved state of a judged proposal
struct LearnBufs {
    uint16_t* X = nullptr;  // [n][48] features
    float* Y = nullptr;     // [n][2] proposals
    float* H = nullptr;     // [n] h_i
    void *px = nullptr, *py = nullptr;                      // positions by id
    void *qx = nullptr, *qy = nullptr;                      // positions by id before the last iteration
    bool have_q = false;
    // two saved cur states: the start of a proposal and the plain branch
    void *bx[2] = {nullptr, nullptr}, *by[2] = {nullptr, nullptr}, *bdp[2] = {nullptr, nullptr};
    int32_t* bid[2] = {nullptr, nullptr};
    uint8_t* bcls[2] = {nullptr, nullptr};
    uint8_t* rflag = nullptr;  // [parts] restore flags
};

namespace trime {
MlpDev mlp_view(const mlp_s* m);
int* mlp_err(mlp_s* m);
}  // namespace trime

template <typename T>
static T* dalloc(mesh_s* m, size_t count, int& rc) {
    if (rc) return nullptr;
    void* p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
        rc = fail(TRIME_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return nullptr;
    }
    m->allocs.push_back(p);
    return static_cast<T*>(p);
}

// ------------------------------------------------------------------ host geometry
static double host_bilin(const mesh_grid2d& g, double dx, double dy, double x, double y) {
    double tx = (x - g.x0) / dx, ty = (y - g.y0) / dy;
    double fi = std::floor(tx), fj = std::floor(ty);
    int i = !(fi >= 0.0) ? 0 : (fi > (double)(g.nx - 2) ? g.nx - 2 : (int)fi);
    int j = !(fj >= 0.0) ? 0 : (fj > (double)(g.ny - 2) ? g.ny - 2 : (int)fj);
    double fx = tx - (double)i, fy = ty - (double)j;
    fx = fx < 0.0 ? 0.0 : (fx > 1.0 ? 1.0 : fx);
    fy = fy < 0.0 ? 0.0 : (fy > 1.0 ? 1.0 : fy);
    const float* r0 = g.v + (size_t)j * g.nx + i;
    const float* r1 = r0 + g.nx;
    double v00 = r0[0], v10 = r0[1], v01 = r1[0], v11 = r1[1];
    double a = v00 + fx * (v10 - v00);
    double b = v01 + fx * (v11 - v01);
    return a + fy * (b - a);
}

static bool grid_ok(const mesh_grid2d* g) {
    if (!g || !g->v || g->nx < 2 || g->ny < 2 || !(g->x1 > g->x0) || !(g->y1 > g->y0)) return false;
    if (!std::isfinite(g->x0) || !std::isfinite(g->x1) || !std::isfinite(g->y0) || !std::isfinite(g->y1)) return false;
    size_t n = (size_t)g->nx * (size_t)g->ny;
    for (size_t k = 0; k < n; k++)
        if (!std::isfinite(g->v[k])) return false;
    return true;
}

struct HostGeometry {
    std::vector<uint8_t> cls, idist, sel;
    std::vector<double> h, geps, rho;
    double sum_rho = 0;
    double havg = 0;
    double rho_eff = 0;  // point-weighted mean point density (points per unit area)
};

// Sec. 3.2 classes from the SDF at cell midpoints; Sec. 3.5 normalised
// density over inner and selected-boundary cells; Sec. 3.7 h_i, geps_i
static int host_geometry(const mesh_grid2d& sdf, const mesh_grid2d& siz, int64_t N, const mesh_params& P,
                         HostGeometry& G) {
    int ncx = sdf.nx - 1, ncy = sdf.ny - 1;
    size_t nc = (size_t)ncx * (size_t)ncy;
    double dx = (sdf.x1 - sdf.x0) / (double)(sdf.nx - 1), dy = (sdf.y1 - sdf.y0) / (double)(sdf.ny - 1);
    double hdx = (siz.x1 - siz.x0) / (double)(siz.nx - 1), hdy = (siz.y1 - siz.y0) / (double)(siz.ny - 1);
    double ldiag = std::sqrt(dx * dx + dy * dy);
    double band = P.eta * std::min(dx, dy);
    G.cls.resize(nc);
    G.h.resize(nc);
    G.geps.resize(nc);
    std::vector<double>& rho = G.rho;
    std::vector<uint8_t>& sel = G.sel;
    rho.assign(nc, 0.0);
    sel.assign(nc, 0);
    double sum_rho = 0.0;
    int64_t nsel = 0;
    for (int gj = 0; gj < ncy; gj++)
        for (int gi = 0; gi < ncx; gi++) {
            size_t c = (size_t)gj * ncx + gi;
            const float* r0 = sdf.v + (size_t)gj * sdf.nx + gi;
            const float* r1 = r0 + sdf.nx;
            double sm = 0.25 * ((((double)r0[0] + (double)r0[1]) + (double)r1[0]) + (double)r1[1]);
            uint8_t k = std::fabs(sm) <= ldiag ? CELL_BOUNDARY : (sm < 0.0 ? CELL_INNER : CELL_OUTER);
            G.cls[c] = k;
            double mx = sdf.x0 + ((double)gi + 0.5) * dx, my = sdf.y0 + ((double)gj + 0.5) * dy;
            double mu = host_bilin(siz, hdx, hdy, mx, my);
            rho[c] = 1.0 / (mu * mu);
            sel[c] = (k == CELL_INNER) || (k == CELL_BOUNDARY && sm <= band);
            if (sel[c]) {
                sum_rho += rho[c];
                nsel++;
            }
        }
    if (nsel == 0) return fail(TRIME_EINVAL, "the SDF grid has no inner or selected boundary cells");
    G.sum_rho = sum_rho;
    double sum_h = 0.0;
    for (int gj = 0; gj < ncy; gj++)
        for (int gi = 0; gi < ncx; gi++) {
            size_t c = (size_t)gj * ncx + gi;
            double nE = (rho[c] / sum_rho) * (double)N;
            G.h[c] = std::sqrt((dx * dy) / nE);
            if (sel[c]) sum_h += G.h[c];
        }
    G.havg = sum_h / (double)nsel;
    for (size_t c = 0; c < nc; c++) G.geps[c] = P.fac_geps * std::min(G.h[c], G.havg);
    // expected point density of cell c is nE_c / (dx dy) = 1 / h_c^2; weighted
    // by the points it holds: sum h^-4 / sum h^-2 over the selected cells
    double s2 = 0.0, s4 = 0.0;
    for (size_t c = 0; c < nc; c++)
        if (sel[c] && std::isfinite(G.h[c]) && G.h[c] > 0) {
            double r = 1.0 / (G.h[c] * G.h[c]);
            s2 += r;
            s4 += r * r;
        }
    G.rho_eff = s2 > 0 ? s4 / s2 : 0.0;
    // Chebyshev distance to the nearest non-inner cell (outside the grid counts)
    std::vector<int> d(nc);
    for (int gj = 0; gj < ncy; gj++)
        for (int gi = 0; gi < ncx; gi++) {
            size_t c = (size_t)gj * ncx + gi;
            int e = std::min(std::min(gi + 1, gj + 1), std::min(ncx - gi, ncy - gj));
            d[c] = G.cls[c] == CELL_INNER ? e : 0;
        }
    for (int gj = 0; gj < ncy; gj++)
        for (int gi = 0; gi < ncx; gi++) {
            size_t c = (size_t)gj * ncx + gi;
            for (int oj = -1; oj <= 0; oj++)
                for (int oi = -1; oi <= 1; oi++) {
                    if (oj == 0 && oi >= 0) continue;
                    int a = gi + oi, b = gj + oj;
                    if (a < 0 || a >= ncx || b < 0) continue;
                    d[c] = std::min(d[c], d[(size_t)b * ncx + a] + 1);
                }
        }
    for (int gj = ncy - 1; gj >= 0; gj--)
        for (int gi = ncx - 1; gi >= 0; gi--) {
            size_t c = (size_t)gj * ncx + gi;
            for (int oj = 0; oj <= 1; oj++)
                for (int oi = -1; oi <= 1; oi++) {
                    if (oj == 0 && oi <= 0) continue;
                    int a = gi + oi, b = gj + oj;
                    if (a < 0 || a >= ncx || b >= ncy) continue;
                    d[c] = std::min(d[c], d[(size_t)b * ncx + a] + 1);
                }
        }
    G.idist.resize(nc);
    for (size_t c = 0; c < nc; c++) G.idist[c] = (uint8_t)std::min(d[c], 255);
    return 0;
}

// ------------------------------------------------------------------ layout
// neighbour buckets: the paper sizes the block grid for N_opt points per
// block under uniform density (Sec. 3.2); with adaptive density we size it so
// that the bucket holding a typical point expects nopt points
static void size_buckets(Part& p, double nopt) {
    DevParams& d = p.dp;
    double W = d.bx1 - d.bx0, H = d.by1 - d.by0;
    int64_t n = p.n;
    double lam = std::sqrt((double)std::max<int64_t>(n, 1) / (nopt * W * H));
    if (p.rho_eff > 0 && n > 0) lam = std::max(lam, std::sqrt(p.rho_eff / nopt));
    double cap = std::sqrt((4.0 * (double)n + 1024.0) / (W * H));
    lam = std::min(lam, cap);
    d.nbx = std::max(1, (int)std::ceil(lam * W));
    d.nby = std::max(1, (int)std::ceil(lam * H));
    d.bsx = W / d.nbx;
    d.bsy = H / d.nby;
    d.bx0f = (float)d.bx0;
    d.by0f = (float)d.by0;
    d.ibsxf = (float)(1.0 / d.bsx);
    d.ibsyf = (float)(1.0 / d.bsy);
    d.Wf = (float)(d.bx1 - d.bx0);
    d.Hf = (float)(d.by1 - d.by0);
    d.bsxf = (float)d.bsx;
    d.bsyf = (float)d.bsy;
    d.bmargf = (float)(1e-3 * (d.bsx > d.bsy ? d.bsx : d.bsy));
    p.nb = d.nbx * d.nby;
}

// bucket offsets of every part; a batch gives each part one pad bucket
static int layout_buckets(mesh_s* m, double nopt) {
    int64_t tot = 0;
    for (Part& p : m->parts) {
        size_buckets(p, nopt);
        p.boff = (int32_t)tot;
        tot += p.nb + (m->batched ? 1 : 0);
    }
    if (tot > (int64_t)1 << 30) return fail(TRIME_EINVAL, "too many buckets");
    m->nbtot = (int)tot;
    m->nopt = nopt;
    return 0;
}

static MeshView view_of(const mesh_s* m, int k) {
    const Part& p = m->parts[k];
    MeshView V;
    std::memset(&V, 0, sizeof V);
    V.P = p.dp;
    V.sdf = p.sdf;
    V.siz = p.siz;
    V.gcls = p.gcls;
    V.gh = p.gh;
    V.ggeps = p.ggeps;
    V.gidist = p.gidist;
    V.ctrl = m->ctrl + k;
    V.soff = p.soff;
    V.n = (int32_t)p.n;
    V.boff = p.boff;
    V.nb = p.nb;
    V.c0 = p.c0;
    V.c1 = p.c1;
    V.npad = p.npad;
    return V;
}

// device table of the views (batch only), after any change of the layout
static int upload_views(mesh_s* m) {
    if (!m->batched) return 0;
    std::vector<MeshView> v(m->parts.size());
    for (size_t k = 0; k < v.size(); k++) v[k] = view_of(m, (int)k);
    CUDA_TRY(cudaMemcpyAsync(m->dviews, v.data(), v.size() * sizeof(MeshView), cudaMemcpyHostToDevice, m->st));
    CUDA_TRY(cudaStreamSynchronize(m->st));
    return 0;
}

// ------------------------------------------------------------------ enqueue helpers
template <typename T>
static IterArgs<T> make_args(mesh_s* m, int force) {
    IterArgs<T> a;
    std::memset(&a, 0, sizeof a);
    a.n = (int32_t)m->nslots;
    a.force = force;
    a.nmesh = (int32_t)m->parts.size();
    a.nbtot = m->nbtot;
    a.V = view_of(m, 0);
    a.Vs = m->batched ? m->dviews : nullptr;
    a.cmesh = m->batched ? m->cmesh : nullptr;
    a.ovf_n = m->ovf_n;
    a.cur = {(T*)m->cx, (T*)m->cy, m->cid, m->ccls, (T*)m->cdp};
    a.srt = {(T*)m->sx, (T*)m->sy, m->sid, m->scls, (T*)m->sdp};
    a.wrk = {(T*)m->wx, (T*)m->wy, m->sid, m->wcls, (T*)m->wdp};
    a.cell = m->cell;
    a.key = m->key;
    a.rank = m->rank;
    a.sidx = m->sidx;
    a.skey = m->skey;
    a.dom = m->dom;
    a.bcount = m->bcount;
    a.bstart = m->bstart;
    a.scan_tmp = m->scan_tmp;
    a.ring = m->ring;
    a.ring_n = m->ring_n;
    a.warm = m->warm;
    a.perm = m->perm;
    a.cellR = m->cellR;
    a.vmask = m->vmask;
    a.ep = m->ep;
    a.up = m->up;
    a.dbg = m->dbg;
    a.ovf_list = m->ovf_list;
    a.ovf2_list = m->ovf_list + std::max<int64_t>(m->ncap, m->nslots);
    a.ovf3_list = m->batched ? nullptr : m->ovf_list + 2 * std::max<int64_t>(m->ncap, m->nslots);
    a.ovf0_list = m->ovf_list + 3 * std::max<int64_t>(m->ncap, m->nslots);
    a.pf = m->pf;
    a.pf3 = m->pf3;
    a.pS = m->pS;
    return a;
}

template <typename T>
static void enqueue_rebuild(mesh_s* m, int force, int decide) {
    IterArgs<T> a = make_args<T>(m, force);
    launch_bucket<T>(a, m->st);
    launch_voronoi<T>(a, m->lanes, m->st);
    launch_emit<T>(a, m->nblk, m->st);
    launch_stats_pre<T>(a, decide, m->st);
}

template <typename T>
static void enqueue_iteration(mesh_s* m) {
    IterArgs<T> a = make_args<T>(m, 0);
    launch_bucket<T>(a, m->st);
    launch_voronoi<T>(a, m->lanes, m->st);
    launch_emit<T>(a, m->nblk, m->st);
    launch_dm_keep<T>(a, m->nblk, m->st);  // runs instead of the three above when the triangulation is kept
    launch_stats_pre<T>(a, 1, m->st);
    launch_update<T>(a, m->nblk, m->st);
    launch_stats_post<T>(a, m->st);
}

static void enqueue(mesh_s* m, bool iteration, int force) {
    if (m->prec == 0) {
        if (iteration) enqueue_iteration<double>(m);
        else enqueue_rebuild<double>(m, force, 0);
    } else {
        if (iteration) enqueue_iteration<float>(m);
        else enqueue_rebuild<float>(m, force, 0);
    }
}

static int sync_in(mesh_s* m) {
    CUDA_TRY(cudaEventRecord(m->ev, m->user));
    CUDA_TRY(cudaStreamWaitEvent(m->st, m->ev, 0));
    return 0;
}

static int sync_out(mesh_s* m) {
    CUDA_TRY(cudaEventRecord(m->ev, m->st));
    CUDA_TRY(cudaStreamWaitEvent(m->user, m->ev, 0));
    return 0;
}

static int read_ctrl(mesh_s* m) {
    CUDA_TRY(cudaMemcpyAsync(m->hctrl, m->ctrl, sizeof(DevCtrl) * m->parts.size(), cudaMemcpyDeviceToHost, m->st));
    CUDA_TRY(cudaStreamSynchronize(m->st));
    return 0;
}

static bool all_terminated(const mesh_s* m) {
    for (size_t k = 0; k < m->parts.size(); k++)
        if (!m->hctrl[k].terminated) return false;
    return true;
}

static void fill_stats(const mesh_s* m, int k, int iters, mesh_stats* s) {
    const DevCtrl& c = m->hctrl[k];
    std::memset(s, 0, sizeof *s);
    s->iterations = iters;
    s->terminated = c.terminated;
    s->method = c.last_method;
    s->switched = c.switched;
    s->n_tri = (int64_t)c.n_tri;
    s->n_edges = (int64_t)c.n_edges;
    s->half_mean_alpha = c.half_a;
    s->half_mean_beta = c.half_b;
    s->max_alpha = c.max_a;
    s->max_beta = c.max_b;
    s->min_angle_deg = c.min_ang;
    s->mean_size_dev = c.size_dev;
    s->fac_mu = c.fac_mu;
    s->exact_calls = (int64_t)c.cnt.exact_calls;
    s->clip_inconsistent = (int64_t)c.cnt.clip_inconsistent;
    s->ring_overflow = (int64_t)c.cnt.ring_overflow;
    s->exact_overflow = (int64_t)c.cnt.exact_overflow;
    s->newton_fail = (int64_t)c.cnt.newton_fail;
    s->trace_cap = (int64_t)c.cnt.trace_cap;
    s->quad_cap = (int64_t)c.cnt.quad_cap;
    s->dup_points = (int64_t)c.cnt.dup_points;
    s->small_moves = c.small_moves;
    s->target_reached = c.target_reached;
    s->vor_candidates = (int64_t)c.cnt.vor_candidates;
    s->vor_picks = (int64_t)c.cnt.vor_picks;
    s->vor_cuts = (int64_t)c.cnt.vor_cuts;
    s->vor_rings = (int64_t)c.cnt.vor_rings;
    s->vor_wide = (int64_t)c.cnt.vor_wide;
    s->triangulations = (int64_t)c.cnt.triangulations;
    s->vor_fp64 = (int64_t)c.cnt.vor_fp64;
    s->vor_resolve = (int64_t)c.cnt.vor_resolve;
    s->vor_direct = (int64_t)c.cnt.vor_direct;
    s->added = m->batched ? 0 : m->added_call;
    s->n_points = m->parts[k].n;
}

static bool guard_tripped(const mesh_s* m) {
    unsigned long long ro = 0, eo = 0;
    for (size_t k = 0; k < m->parts.size(); k++) {
        ro += m->hctrl[k].cnt.ring_overflow;
        eo += m->hctrl[k].cnt.exact_overflow;
    }
    if (!ro && !eo) return false;
    fail(TRIME_EDEVICE, "capacity guard tripped: " + std::to_string(ro) + " cells with more than 64 edges, " +
                            std::to_string(eo) + " exact-arithmetic capacity or underflow guards");
    return true;
}

__global__ void k_reset_counters(DevCtrl* ctrl, int n) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) ctrl[k].cnt = DevCounters{};
}

// the next iteration of part k (all parts for k < 0) re-triangulates: the
// sorted order or the positions changed outside an iteration
__global__ void k_force_retri(DevCtrl* ctrl, int lo, int hi) {
    int k = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (k < hi) ctrl[k].retri = 1;
}

static int force_retri(mesh_s* m, int k) {
    int lo = k < 0 ? 0 : k, hi = k < 0 ? (int)m->parts.size() : k + 1;
    k_force_retri<<<(hi - lo + 127) / 128, 128, 0, m->st>>>(m->ctrl, lo, hi);
    CUDA_TRY(cudaGetLastError());
    return 0;
}

static int reset_counters(mesh_s* m) {
    int n = (int)m->parts.size();
    k_reset_counters<<<(n + 127) / 128, 128, 0, m->st>>>(m->ctrl, n);
    CUDA_TRY(cudaGetLastError());
    return 0;
}

// ------------------------------------------------------------------ creation
static int check_params(const mesh_params& P) {
    if (P.precision != 0 && P.precision != 1) return fail(TRIME_EINVAL, "precision must be 0 or 1");
    if (P.method < 0 || P.method > 2) return fail(TRIME_EINVAL, "method must be 0, 1 or 2");
    if (P.quad_max_level < 1 || P.quad_max_level > 9) return fail(TRIME_EINVAL, "quad_max_level must be 1..9");
    if (P.newton_max < 0 || P.trace_max < 1) return fail(TRIME_EINVAL, "bad newton_max / trace_max");
    if (!(P.N_opt > 0) || !(P.fac_voro_bound > 0) || !(P.dt >= 0)) return fail(TRIME_EINVAL, "bad parameter value");
    if (!(P.fac_add > 0) || !(P.T_add >= 0) || P.n_total < 0 || P.n_total > (int64_t)(1 << 30))
        return fail(TRIME_EINVAL, "bad point-addition parameter (fac_add > 0, T_add >= 0, 0 <= n_total <= 2^30)");
    return 0;
}

static int check_part(const mesh_grid2d* sdf, const mesh_grid2d* sizing, const void* xy, int64_t n, int prec,
                      const std::string& who) {
    if (n < 0 || n > (int64_t)(1 << 30)) return fail(TRIME_EINVAL, who + "n out of range");
    if (n > 0 && !xy) return fail(TRIME_EINVAL, who + "xy is NULL");
    if (!grid_ok(sdf)) return fail(TRIME_EINVAL, who + "invalid SDF grid");
    if (!grid_ok(sizing)) return fail(TRIME_EINVAL, who + "invalid sizing grid");
    for (size_t k = 0; k < (size_t)sizing->nx * sizing->ny; k++)
        if (!(sizing->v[k] > 0.0f)) return fail(TRIME_EINVAL, who + "sizing values must be positive");
    for (int64_t i = 0; i < n; i++) {
        double x = prec == 0 ? ((const double*)xy)[2 * i] : (double)((const float*)xy)[2 * i];
        double y = prec == 0 ? ((const double*)xy)[2 * i + 1] : (double)((const float*)xy)[2 * i + 1];
        if (!std::isfinite(x) || !std::isfinite(y) || x < sdf->x0 || x > sdf->x1 || y < sdf->y0 || y > sdf->y1)
            return fail(TRIME_EINVAL,
                        who + "point " + std::to_string(i) + " is not finite or outside the SDF grid box");
    }
    return 0;
}

static DevGrid dev_grid(const mesh_grid2d* g, const float* dv) {
    DevGrid d{g->nx, g->ny, g->x0, g->y0, g->x1, g->y1, (g->x1 - g->x0) / (double)(g->nx - 1),
              (g->y1 - g->y0) / (double)(g->ny - 1), dv, 0.0, 0.0};
    d.idx = 1.0 / d.dx;
    d.idy = 1.0 / d.dy;
    auto split = [](double v, float& h, float& l) {
        h = (float)v;
        l = (float)(v - (double)h);
    };
    split(d.x0, d.fx0h, d.fx0l);
    split(d.y0, d.fy0h, d.fy0l);
    split(d.idx, d.fidxh, d.fidxl);
    split(d.idy, d.fidyh, d.fidyl);
    return d;
}

static void fill_devparams(DevParams& d, const mesh_params& P, const HostGeometry& G, const mesh_grid2d* sdf) {
    std::memset(&d, 0, sizeof d);
    d.bounded = P.bounded;
    d.validity = P.validity;
    d.newton_max = P.newton_max;
    d.trace_max = P.trace_max;
    d.quad_max_level = P.quad_max_level;
    d.debug = P.debug != 0;
    d.fac_F = P.fac_F;
    d.k_spring = P.k_spring;
    d.dt = P.dt;
    d.fac_pt = P.fac_pt;
    d.fac_geps = P.fac_geps;
    d.fac_voro_bound = P.fac_voro_bound;
    d.fac_end = P.fac_end;
    d.T_circ = P.T_circ;
    d.T_switch = P.T_switch;
    d.T_end_q = P.T_end_q;
    d.T_end_amax = P.T_end_amax;
    d.damping = P.damping;
    d.fac_retria = P.fac_retria;
    d.T_add = P.T_add;
    d.havg = G.havg;
    d.bx0 = sdf->x0;
    d.by0 = sdf->y0;
    d.bx1 = sdf->x1;
    d.by1 = sdf->y1;
}

// uploads part k's grids and initial state (ids soff + i in input order,
// classes by Sec. 4.3 on the host)
static int upload_part(mesh_s* m, int k, const mesh_grid2d* sdf, const mesh_grid2d* sizing, const void* xy,
                       const HostGeometry& G) {
    Part& p = m->parts[k];
    size_t N = (size_t)p.n, T = m->prec == 0 ? sizeof(double) : sizeof(float);
    size_t ns = (size_t)sdf->nx * sdf->ny, nz = (size_t)sizing->nx * sizing->ny;
    size_t nc = (size_t)(sdf->nx - 1) * (sdf->ny - 1);
    int rc = 0;
    float* dsdf = dalloc<float>(m, ns, rc);
    float* dsiz = dalloc<float>(m, nz, rc);
    p.gcls = dalloc<uint8_t>(m, nc, rc);
    p.gh = dalloc<double>(m, nc, rc);
    p.ggeps = dalloc<double>(m, nc, rc);
    p.gidist = dalloc<uint8_t>(m, nc, rc);
    if (rc) return rc;
    p.sdf = dev_grid(sdf, dsdf);
    p.siz = dev_grid(sizing, dsiz);
    auto H2D = [&](void* dst, const void* src, size_t bytes) {
        return bytes == 0 || cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, m->st) == cudaSuccess;
    };
    bool ok = H2D(dsdf, sdf->v, ns * sizeof(float)) && H2D(dsiz, sizing->v, nz * sizeof(float)) &&
              H2D(p.gcls, G.cls.data(), nc) && H2D(p.gh, G.h.data(), nc * sizeof(double)) &&
              H2D(p.ggeps, G.geps.data(), nc * sizeof(double)) && H2D(p.gidist, G.idist.data(), nc);
    std::vector<int32_t> ids(N);
    std::vector<uint8_t> cls(N);
    std::vector<char> dp(N * T), xs(N * T), ys(N * T);
    double sdx = p.sdf.dx, sdy = p.sdf.dy;
    int ncx = sdf->nx - 1, ncy = sdf->ny - 1;
    for (size_t i = 0; i < N; i++) {
        ids[i] = p.soff + (int32_t)i;
        double x = m->prec == 0 ? ((const double*)xy)[2 * i] : (double)((const float*)xy)[2 * i];
        double y = m->prec == 0 ? ((const double*)xy)[2 * i + 1] : (double)((const float*)xy)[2 * i + 1];
        double fi = std::floor((x - sdf->x0) / sdx), fj = std::floor((y - sdf->y0) / sdy);
        bool inside = fi >= 0 && fi <= ncx - 1 && fj >= 0 && fj <= ncy - 1;
        int gi = !(fi >= 0) ? 0 : (fi > ncx - 1 ? ncx - 1 : (int)fi);
        int gj = !(fj >= 0) ? 0 : (fj > ncy - 1 ? ncy - 1 : (int)fj);
        size_t c = (size_t)gj * ncx + gi;
        uint8_t pc = PT_BOUNDARY;
        if (inside && G.cls[c] == CELL_INNER) pc = PT_INNER;
        else if (inside && G.cls[c] == CELL_BOUNDARY) {
            double s = host_bilin(*sdf, sdx, sdy, x, y);
            if (s < -G.geps[c]) pc = PT_INNER;
        }
        cls[i] = pc;  // reading: a point outside at init counts as boundary
        double h = G.h[c];
        if (m->prec == 0) {
            ((double*)xs.data())[i] = x;
            ((double*)ys.data())[i] = y;
            ((double*)dp.data())[i] = h;  // reading: eps_c = 1 at the first iteration
        } else {
            ((float*)xs.data())[i] = (float)x;
            ((float*)ys.data())[i] = (float)y;
            ((float*)dp.data())[i] = (float)h;
        }
    }
    size_t o = (size_t)p.soff;
    ok = ok && H2D((char*)m->cx + o * T, xs.data(), N * T) && H2D((char*)m->cy + o * T, ys.data(), N * T) &&
         H2D((char*)m->cdp + o * T, dp.data(), N * T) && H2D(m->cid + o, ids.data(), N * sizeof(int32_t)) &&
         H2D(m->ccls + o, cls.data(), N);
    DevCtrl c0;
    std::memset(&c0, 0, sizeof c0);
    c0.method_param = m->P.method;
    c0.last_method = -1;
    c0.retri = 1;
    ok = ok && H2D(m->ctrl + k, &c0, sizeof c0);
    // the host vectors above must outlive the copies
    if (!ok || cudaStreamSynchronize(m->st) != cudaSuccess) return fail(TRIME_ECUDA, "initial upload failed");
    return 0;
}

static int capture_graph(mesh_s* m) {
    if (m->gexec) {
        cudaGraphExecDestroy(m->gexec);
        m->gexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(m->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail(TRIME_ECUDA, "cudaStreamBeginCapture failed");
    enqueue(m, true, 0);
    cudaError_t e = cudaStreamEndCapture(m->st, &graph);
    if (e != cudaSuccess) return fail(TRIME_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&m->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(TRIME_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return 0;
}

// times rebuilds (a1..a4, no move) for each candidate bucket size and Voronoi
// lane count and keeps the fastest; results do not depend on the choice
static int autotune(mesh_s* m, const std::vector<double>& nopts) {
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    const int lanes_c[3] = {8, 16, 32};
    TuneCand best{m->nopt, m->lanes, 1e300};
    m->tune.clear();
    int rc = 0;
    for (double no : nopts) {
        for (int ln : lanes_c) {
            if ((rc = layout_buckets(m, no)) || (rc = upload_views(m))) break;
            m->lanes = ln;
            enqueue(m, false, 1);  // warm-up
            CUDA_TRY(cudaEventRecord(e0, m->st));
            for (int r = 0; r < 2; r++) enqueue(m, false, 1);
            CUDA_TRY(cudaEventRecord(e1, m->st));
            CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0;
            CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            TuneCand c{no, ln, ms * 0.5};
            m->tune.push_back(c);
            if (c.ms < best.ms) best = c;
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    m->lanes = best.lanes;
    if ((rc = layout_buckets(m, best.nopt)) || (rc = upload_views(m))) return rc;
    return reset_counters(m);
}

// shared by mesh_init (one part, no padding) and mesh_batch_init
static int create(mesh_s* m, int nparts, const mesh_grid2d* sdfs, const mesh_grid2d* sizings,
                  const void* const* xys, const int64_t* ns, const mesh_params& P, void* cuda_stream,
                  int tune) {
    int rc = check_params(P);
    if (rc) return rc;
    m->prec = P.precision;
    m->P = P;
    m->user = (cudaStream_t)cuda_stream;
    m->parts.resize(nparts);
    std::vector<HostGeometry> G(nparts);
    int64_t slots = 0;
    for (int k = 0; k < nparts; k++) {
        std::string who = m->batched ? "mesh " + std::to_string(k) + ": " : "";
        if ((rc = check_part(&sdfs[k], &sizings[k], xys ? xys[k] : nullptr, ns[k], P.precision, who))) return rc;
        if (m->batched && P.n_total > ns[k])
            return fail(TRIME_EINVAL, who + "point addition (n_total above n) is not available in a batch");
        if ((rc = host_geometry(sdfs[k], sizings[k], ns[k], P, G[k]))) return fail(rc, who + g_err);
        Part& p = m->parts[k];
        p.n = ns[k];
        fill_devparams(p.dp, P, G[k], &sdfs[k]);
        p.rho_eff = G[k].rho_eff;
        p.soff = (int32_t)slots;
        int64_t len = m->batched ? (p.n + kChunk - 1) / kChunk * kChunk : p.n;
        p.npad = (int32_t)(len - p.n);
        slots += len;
        if (slots > (int64_t)1 << 30) return fail(TRIME_EINVAL, "too many points");
        p.c0 = (int32_t)(p.soff / kChunk);
        p.c1 = (int32_t)((p.soff + len) / kChunk);
    }
    m->nslots = slots;
    m->nblk = m->batched ? (int)(slots / kChunk) : (int)std::max<int64_t>(1, (slots + kThreads - 1) / kThreads);
    if (!m->batched) m->parts[0].c1 = m->nblk;
    // a single mesh holds up to N_total points (Sec. 3.6): device arrays, the
    // bucket grid and the block partials are sized for that many
    m->ncap = m->batched ? slots : std::max<int64_t>(slots, P.n_total);
    if (m->ncap > (int64_t)1 << 30) return fail(TRIME_EINVAL, "too many points");
    for (Part& p : m->parts) p.dp.adding = !m->batched && p.n < m->ncap;
    int nblk_cap = m->batched ? m->nblk : (int)std::max<int64_t>(1, (m->ncap + kThreads - 1) / kThreads);
    std::vector<double> nopts = {P.N_opt};
    if (tune) nopts = {P.N_opt * (2.0 / 3.0), P.N_opt, P.N_opt * 1.5};
    int nbmax = 0;
    for (int at_cap = 0; at_cap < 2; at_cap++) {
        Part& p0 = m->parts[0];
        int64_t n_now = p0.n;
        double rho_now = p0.rho_eff;
        if (at_cap && !m->batched && m->ncap > n_now) {
            // the expected point density grows with N_current (h_i ~ N^-1/2)
            if (n_now > 0) p0.rho_eff = rho_now * ((double)m->ncap / (double)n_now) * (1.0 + 1e-9);
            p0.n = m->ncap;
        }
        for (double no : nopts) {
            if ((rc = layout_buckets(m, no))) return rc;
            nbmax = std::max(nbmax, m->nbtot);
        }
        p0.n = n_now;
        p0.rho_eff = rho_now;
    }

    if (cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev, cudaEventDisableTiming) != cudaSuccess)
        return fail(TRIME_ECUDA, "stream/event creation failed");
    if (cudaMallocHost(&m->hctrl, sizeof(DevCtrl) * nparts) != cudaSuccess) return fail(TRIME_ENOMEM, "pinned alloc");

    size_t N = (size_t)m->ncap;
    size_t T = P.precision == 0 ? sizeof(double) : sizeof(float);
    size_t nmax = 0;
    for (const Part& p : m->parts) nmax = std::max(nmax, (size_t)p.n);
    if (!m->batched) nmax = N;
    rc = 0;
    m->cx = dalloc<char>(m, N * T, rc);
    m->cy = dalloc<char>(m, N * T, rc);
    m->cdp = dalloc<char>(m, N * T, rc);
    m->sx = dalloc<char>(m, N * T, rc);
    m->sy = dalloc<char>(m, N * T, rc);
    m->sdp = dalloc<char>(m, N * T, rc);
    m->wx = dalloc<char>(m, N * T, rc);
    m->wy = dalloc<char>(m, N * T, rc);
    m->wdp = dalloc<char>(m, N * T, rc);
    m->wcls = dalloc<uint8_t>(m, N, rc);
    m->cid = dalloc<int32_t>(m, N, rc);
    m->sid = dalloc<int32_t>(m, N, rc);
    m->ccls = dalloc<uint8_t>(m, N, rc);
    m->scls = dalloc<uint8_t>(m, N, rc);
    m->cell = dalloc<int32_t>(m, N, rc);
    m->key = dalloc<int32_t>(m, N, rc);
    m->rank = dalloc<int32_t>(m, N, rc);
    m->sidx = dalloc<int32_t>(m, N, rc);
    m->skey = dalloc<int32_t>(m, N, rc);
    m->dom = dalloc<uint8_t>(m, N, rc);
    m->bcount = dalloc<int32_t>(m, (size_t)nbmax, rc);
    m->bstart = dalloc<int32_t>(m, (size_t)nbmax + 1, rc);
    size_t scan_n = std::max<size_t>((size_t)nbmax + 1, N + 1);
    m->scan_tmp = dalloc<int32_t>(m, scan_n / 4096 + 2, rc);
    m->nbcap = nbmax;
    m->ring = dalloc<int32_t>(m, N * kRingCap, rc);
    m->ring_n = dalloc<uint8_t>(m, N, rc);
    m->warm = dalloc<int32_t>(m, N * kWarm, rc);
    m->perm = dalloc<int32_t>(m, N, rc);
    m->cellR = dalloc<float>(m, N, rc);
    m->vmask = dalloc<uint64_t>(m, N, rc);
    m->ep = dalloc<EmitPartial>(m, (size_t)nblk_cap, rc);
    m->up = dalloc<UpdatePartial>(m, (size_t)nblk_cap, rc);
    m->ctrl = dalloc<DevCtrl>(m, (size_t)nparts, rc);
    m->ovf_n = dalloc<int32_t>(m, 4, rc);
    m->chk = dalloc<int32_t>(m, 1, rc);
    if (!rc && cudaMallocHost(&m->hchk, sizeof(int32_t)) != cudaSuccess) rc = fail(TRIME_ENOMEM, "pinned alloc");
    m->dbg = P.debug ? dalloc<double>(m, 10 * N, rc) : nullptr;
    m->tcnt = dalloc<int32_t>(m, N + 1, rc);
    m->toff = dalloc<int32_t>(m, N + 1, rc);
    m->tbuf = dalloc<int32_t>(m, 3 * (2 * nmax + 16), rc);
    m->xybuf = dalloc<char>(m, 2 * N * std::max<size_t>(T, sizeof(double)), rc);
    m->ovf_list = dalloc<int32_t>(m, 4 * N, rc);
    m->pf = dalloc<float4>(m, N, rc);
    m->pf3 = dalloc<float2>(m, N, rc);
    m->pS = dalloc<float>(m, N, rc);
    if (m->batched) {
        m->dviews = dalloc<MeshView>(m, (size_t)nparts, rc);
        m->cmesh = dalloc<int32_t>(m, N / kChunk, rc);
    }
    if (!m->batched && m->ncap > slots) {
        m->akeys = dalloc<char>(m, (2 * N + 16) * kAddKeyBytes, rc);
        m->ahist = dalloc<int32_t>(m, 256, rc);
        m->acnt = dalloc<int32_t>(m, N + 1, rc);
        m->aoff = dalloc<int32_t>(m, N + 1, rc);
        if (!rc && cudaMallocHost(&m->hhist, 256 * sizeof(int32_t)) != cudaSuccess)
            rc = fail(TRIME_ENOMEM, "pinned alloc");
    }
    if (rc) return rc;
    // padding slots hold zeros; no kernel reads them as points
    CUDA_TRY(cudaMemsetAsync(m->cx, 0, N * T, m->st));
    CUDA_TRY(cudaMemsetAsync(m->cy, 0, N * T, m->st));
    CUDA_TRY(cudaMemsetAsync(m->cdp, 0, N * T, m->st));
    CUDA_TRY(cudaMemsetAsync(m->cid, 0, N * sizeof(int32_t), m->st));
    CUDA_TRY(cudaMemsetAsync(m->ccls, 0, N, m->st));
    CUDA_TRY(cudaMemsetAsync(m->ring_n, 0, N, m->st));  // no previous triangulation
    for (int k = 0; k < nparts; k++)
        if ((rc = upload_part(m, k, &sdfs[k], &sizings[k], xys ? xys[k] : nullptr, G[k]))) return rc;
    if (m->batched) {
        std::vector<int32_t> cm(N / kChunk);
        for (int k = 0; k < nparts; k++)
            for (int32_t c = m->parts[k].c0; c < m->parts[k].c1; c++) cm[c] = k;
        if (!cm.empty()) CUDA_TRY(cudaMemcpyAsync(m->cmesh, cm.data(), cm.size() * 4, cudaMemcpyHostToDevice, m->st));
        CUDA_TRY(cudaStreamSynchronize(m->st));
    }
    if ((rc = layout_buckets(m, P.N_opt)) || (rc = upload_views(m))) return rc;
    if (tune && (rc = autotune(m, nopts))) return rc;
    return capture_graph(m);
}

// ------------------------------------------------------------------ operations shared by both handles
static void destroy(mesh_s* m) {
    if (m->st) cudaStreamSynchronize(m->st);
    delete m->learn;
    if (m->qs) {
        if (m->qs->b.hhist) cudaFreeHost(m->qs->b.hhist);
        delete m->qs;
    }
    if (m->gexec) cudaGraphExecDestroy(m->gexec);
    for (void* p : m->allocs) cudaFree(p);
    if (m->hctrl) cudaFreeHost(m->hctrl);
    if (m->hhist) cudaFreeHost(m->hhist);
    if (m->hchk) cudaFreeHost(m->hchk);
    if (m->ev) cudaEventDestroy(m->ev);
    if (m->st) cudaStreamDestroy(m->st);
}

// stats: one entry per part, or NULL
static int do_rebuild(mesh_s* m, mesh_stats* stats) {
    int rc = sync_in(m);
    if (rc) return rc;
    if ((rc = reset_counters(m))) return rc;
    enqueue(m, false, 1);
    if ((rc = force_retri(m, -1))) return rc;  // cur keeps the previous sorted order
    m->tri_stale = false;
    CUDA_TRY(cudaGetLastError());
    if ((rc = read_ctrl(m))) return rc;
    if ((rc = sync_out(m))) return rc;
    if (stats)
        for (size_t k = 0; k < m->parts.size(); k++) fill_stats(m, (int)k, 0, &stats[k]);
    if (guard_tripped(m)) return TRIME_EDEVICE;
    return TRIME_OK;
}

// Sec. 3.6 point addition on a single mesh whose graph paused for it
// (ctrl->terminated == 2): selection, numbering and the new points on the
// device (addition.cu), the Sec. 3.7 rescaling of h_i, geps_i, h_avg and the
// bucket density, then the layout and the captured iteration for the new
// size.  The paused iteration's triangulation is read in place.
static int add_points(mesh_s* m) {
    Part& p = m->parts[0];
    const int64_t n0 = p.n;
    int64_t nadd = (int64_t)std::floor(m->P.fac_add * (double)n0);
    nadd = std::min<int64_t>(std::max<int64_t>(nadd, 1), m->ncap - n0);
    if (nadd <= 0 || !m->akeys) return fail(TRIME_EDEVICE, "point addition requested without room for points");
    int32_t ntri = 0;
    if (m->prec == 0) launch_tri_count<double>(make_args<double>(m, 1), 0, (int32_t)n0, m->tcnt, m->st);
    else launch_tri_count<float>(make_args<float>(m, 1), 0, (int32_t)n0, m->tcnt, m->st);
    launch_scan(m->tcnt, m->toff, (int32_t)n0, m->scan_tmp, m->st);
    CUDA_TRY(cudaMemcpyAsync(&ntri, m->toff + n0, sizeof(int32_t), cudaMemcpyDeviceToHost, m->st));
    CUDA_TRY(cudaStreamSynchronize(m->st));
    if ((size_t)ntri > 2 * (size_t)m->ncap + 16) return fail(TRIME_EDEVICE, "triangle count exceeds 2n+16");
    nadd = std::min<int64_t>(nadd, ntri);
    if (nadd <= 0) return fail(TRIME_EDEVICE, "point addition requested on a mesh without triangles");
    const int64_t n1 = n0 + nadd;
    const double scale = std::sqrt((double)n0 / (double)n1);
    int32_t nc = (int32_t)((size_t)(p.sdf.nx - 1) * (size_t)(p.sdf.ny - 1));
    std::string err;
    int r = m->prec == 0 ? add_select<double>(make_args<double>(m, 1), (int32_t)n0, ntri, nadd, m->toff, m->akeys,
                                              m->ahist, m->hhist, m->acnt, m->aoff, m->scan_tmp, p.gh, p.ggeps, nc,
                                              scale, m->st, err)
                         : add_select<float>(make_args<float>(m, 1), (int32_t)n0, ntri, nadd, m->toff, m->akeys,
                                             m->ahist, m->hhist, m->acnt, m->aoff, m->scan_tmp, p.gh, p.ggeps, nc,
                                             scale, m->st, err);
    if (r) return fail(r == -1 ? TRIME_ECUDA : TRIME_EDEVICE, err);
    // Sec. 3.7: the quantities scale with sqrt(N_old / N_current); the
    // expected point density (bucket sizing) with N_current / N_old
    p.dp.havg *= scale;
    p.rho_eff *= (double)n1 / (double)n0;
    p.n = n1;
    p.dp.adding = n1 < m->ncap;
    m->nslots = n1;
    m->nblk = (int)std::max<int64_t>(1, (n1 + kThreads - 1) / kThreads);
    p.c1 = m->nblk;
    int rc = layout_buckets(m, m->nopt);
    if (rc) return rc;
    if (m->nbtot > m->nbcap) return fail(TRIME_EDEVICE, "bucket grid outgrew its allocation");
    // the paused iteration counted; the next one re-triangulates and measures
    // no quality change across the addition
    DevCtrl& c = m->hctrl[0];
    c.terminated = 0;
    c.have_prev = 0;
    c.retri = 1;
    c.moved_far = 0;
    CUDA_TRY(cudaMemcpyAsync(m->ctrl, &c, sizeof(DevCtrl), cudaMemcpyHostToDevice, m->st));
    CUDA_TRY(cudaStreamSynchronize(m->st));
    m->tri_stale = true;
    m->added_call += nadd;
    return capture_graph(m);
}

static bool growing(const mesh_s* m) { return !m->batched && m->parts[0].n < m->ncap; }

static int do_step(mesh_s* m, int32_t n_iters, mesh_stats* stats) {
    if (n_iters < 0) return fail(TRIME_EINVAL, "n_iters < 0");
    if (m->learn && n_iters > 0) m->learn->have_q = false;  // the features' last move is no longer known
    int rc = sync_in(m);
    if (rc) return rc;
    if ((rc = reset_counters(m))) return rc;
    m->added_call = 0;
    if (!stats && !growing(m) && !m->tri_stale) {
        // asynchronous: only enqueue.  A mesh that has terminated (on the
        // device, possibly in an iteration still in flight) turns every later
        // launch of the graph into empty kernels, so no host read is needed.
        // (A stale sorted order needs the host to know whether an iteration
        // will re-triangulate, so that case takes the synchronous path.)
        for (int32_t k = 0; k < n_iters; k++) CUDA_TRY(cudaGraphLaunch(m->gexec, m->st));
        return sync_out(m);
    }
    if ((rc = read_ctrl(m))) return rc;
    // a pause left by an asynchronous call
    if (!m->batched && m->hctrl[0].terminated == 2 && (rc = add_points(m))) return rc;
    size_t np = m->parts.size();
    std::vector<int> start(np);
    for (size_t k = 0; k < np; k++) start[k] = m->hctrl[k].iterations;
    if (growing(m)) {
        // point addition: check for a pause every 8 iterations and count the
        // executed iterations (those after a pause were device-side no-ops)
        int done = 0;
        while (done < n_iters) {
            int chunk = std::min(8, n_iters - done);
            m->tri_stale = false;  // the next iteration re-triangulates
            for (int k = 0; k < chunk; k++) CUDA_TRY(cudaGraphLaunch(m->gexec, m->st));
            if ((rc = read_ctrl(m))) return rc;
            if (m->hctrl[0].terminated == 2 && (rc = add_points(m))) return rc;
            done = m->hctrl[0].iterations - start[0];
            if (m->hctrl[0].terminated) break;
        }
    } else if (!all_terminated(m)) {
        if (n_iters > 0) m->tri_stale = false;  // the first iteration re-triangulates
        for (int32_t k = 0; k < n_iters; k++) {
            CUDA_TRY(cudaGraphLaunch(m->gexec, m->st));
            if ((k & 31) == 31 || (stats && k == n_iters - 1)) {
                if ((rc = read_ctrl(m))) return rc;
                if (all_terminated(m)) break;
            }
        }
    }
    if (!stats) return sync_out(m);  // a growing mesh without stats: no final read-back
    if ((rc = read_ctrl(m))) return rc;
    if ((rc = sync_out(m))) return rc;
    for (size_t k = 0; k < np; k++) fill_stats(m, (int)k, m->hctrl[k].iterations - start[k], &stats[k]);
    if (guard_tripped(m)) return TRIME_EDEVICE;
    return TRIME_OK;
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static int get_triangles(mesh_s* m, int k, int32_t* tri, int64_t cap, int64_t* n_out) {
    const Part& p = m->parts[k];
    int rc = sync_in(m);
    if (rc) return rc;
    if (m->tri_stale) {
        enqueue(m, false, 1);
        if ((rc = force_retri(m, -1))) return rc;
        m->tri_stale = false;
    }
    int32_t total = 0;
    if (p.n > 0) {
        if (m->prec == 0) launch_tri_count<double>(make_args<double>(m, 1), p.soff, (int32_t)p.n, m->tcnt, m->st);
        else launch_tri_count<float>(make_args<float>(m, 1), p.soff, (int32_t)p.n, m->tcnt, m->st);
        launch_scan(m->tcnt, m->toff, (int32_t)p.n, m->scan_tmp, m->st);
        CUDA_TRY(cudaMemcpyAsync(&total, m->toff + p.n, sizeof(int32_t), cudaMemcpyDeviceToHost, m->st));
        CUDA_TRY(cudaStreamSynchronize(m->st));
    }
    *n_out = total;
    if (cap < total) return fail(TRIME_ECAPACITY, "triangle buffer too small");
    if (total == 0) return sync_out(m);
    if (!tri) return fail(TRIME_EINVAL, "tri is NULL");
    bool dev = is_device_ptr(tri);
    int32_t* dst = dev ? tri : m->tbuf;
    if (!dev && (size_t)total > 2 * (size_t)p.n + 16) return fail(TRIME_EDEVICE, "triangle count exceeds 2n+16");
    if (m->prec == 0) launch_tri_write<double>(make_args<double>(m, 1), p.soff, (int32_t)p.n, m->toff, dst, m->st);
    else launch_tri_write<float>(make_args<float>(m, 1), p.soff, (int32_t)p.n, m->toff, dst, m->st);
    if (!dev) {
        CUDA_TRY(cudaMemcpyAsync(tri, dst, sizeof(int32_t) * 3 * (size_t)total, cudaMemcpyDeviceToHost, m->st));
        CUDA_TRY(cudaStreamSynchronize(m->st));
    }
    CUDA_TRY(cudaGetLastError());
    return sync_out(m);
}

static int quality(mesh_s* m, int k, mesh_quality_stats* q) {
    const Part& p = m->parts[k];
    int rc = sync_in(m);
    if (rc) return rc;
    if (m->tri_stale) {
        enqueue(m, false, 1);
        if ((rc = force_retri(m, -1))) return rc;
        m->tri_stale = false;
    }
    if (!m->qs) {
        QualityScratch* Q = new QualityScratch();
        size_t N = (size_t)std::max<int64_t>(m->nslots, m->ncap) + 1;
        Q->cap_t = 2 * (int64_t)N + 16;
        Q->cap_e = 3 * (int64_t)N + 16;
        Q->b.tcnt = dalloc<int32_t>(m, N, rc);
        Q->b.ecnt = dalloc<int32_t>(m, N, rc);
        Q->b.toff = dalloc<int32_t>(m, N, rc);
        Q->b.eoff = dalloc<int32_t>(m, N, rc);
        Q->b.scan_tmp = dalloc<int32_t>(m, N / 4096 + 2, rc);
        Q->b.alpha = dalloc<double>(m, (size_t)Q->cap_t, rc);
        Q->b.beta = dalloc<double>(m, (size_t)Q->cap_t, rc);
        Q->b.ang = dalloc<double>(m, (size_t)Q->cap_t, rc);
        Q->b.dev = dalloc<double>(m, (size_t)Q->cap_e, rc);
        Q->b.part = reinterpret_cast<QPartial*>(dalloc<char>(m, 152 * 256, rc));
        Q->b.hist = dalloc<unsigned int>(m, 256, rc);
        if (!rc && cudaMallocHost(&Q->b.hhist, 256 * sizeof(unsigned int)) != cudaSuccess)
            rc = fail(TRIME_ENOMEM, "pinned alloc");
        if (rc) {
            if (Q->b.hhist) cudaFreeHost(Q->b.hhist);
            delete Q;
            return rc;
        }
        m->qs = Q;
    }
    if ((rc = read_ctrl(m))) return rc;
    std::string err;
    const double fac_mu = m->hctrl[k].fac_mu;
    int r = m->prec == 0 ? quality_report<double>(make_args<double>(m, 1), p.soff, (int32_t)p.n, fac_mu, m->qs->b,
                                                  m->qs->cap_t, m->qs->cap_e, m->st, q, err)
                         : quality_report<float>(make_args<float>(m, 1), p.soff, (int32_t)p.n, fac_mu, m->qs->b,
                                                 m->qs->cap_t, m->qs->cap_e, m->st, q, err);
    if (r) return fail(r == -1 ? TRIME_ECUDA : TRIME_EDEVICE, err);
    return sync_out(m);
}

static int get_points(mesh_s* m, int k, void* xy, int64_t cap, int64_t* n_out) {
    const Part& p = m->parts[k];
    *n_out = p.n;
    if (cap < p.n) return fail(TRIME_ECAPACITY, "point buffer too small");
    if (p.n == 0) return TRIME_OK;
    if (!xy) return fail(TRIME_EINVAL, "xy is NULL");
    int rc = sync_in(m);
    if (rc) return rc;
    size_t T = m->prec == 0 ? sizeof(double) : sizeof(float);
    bool dev = is_device_ptr(xy);
    void* dst = dev ? xy : m->xybuf;
    if (m->prec == 0) launch_unpermute<double>(make_args<double>(m, 1), p.soff, (int32_t)p.n, (double*)dst, m->st);
    else launch_unpermute<float>(make_args<float>(m, 1), p.soff, (int32_t)p.n, (float*)dst, m->st);
    if (!dev) {
        CUDA_TRY(cudaMemcpyAsync(xy, dst, 2 * T * (size_t)p.n, cudaMemcpyDeviceToHost, m->st));
        CUDA_TRY(cudaStreamSynchronize(m->st));
    }
    CUDA_TRY(cudaGetLastError());
    return sync_out(m);
}

static int set_state(mesh_s* m, int k, const void* xy, const uint8_t* cls, const double* dprev) {
    const Part& p = m->parts[k];
    if (p.n == 0) return TRIME_OK;
    size_t N = (size_t)p.n, T = m->prec == 0 ? sizeof(double) : sizeof(float);
    int rc = sync_in(m);
    if (rc) return rc;
    // staging: xy in xybuf, cls in tcnt, dprev in tbuf (all large enough)
    char* sxy = (char*)m->xybuf;
    uint8_t* scls = (uint8_t*)m->tcnt;
    double* sdp = (double*)m->tbuf;
    if (xy) {
        // the positions are checked on the device before anything is changed
        CUDA_TRY(cudaMemcpyAsync(sxy, xy, 2 * N * T, cudaMemcpyHostToDevice, m->st));
        CUDA_TRY(cudaMemsetAsync(m->chk, 0x7f, sizeof(int32_t), m->st));
        if (m->prec == 0)
            launch_check_points<double>((const double*)sxy, (int32_t)N, p.dp.bx0, p.dp.by0, p.dp.bx1, p.dp.by1,
                                        m->chk, m->st);
        else
            launch_check_points<float>((const float*)sxy, (int32_t)N, p.dp.bx0, p.dp.by0, p.dp.bx1, p.dp.by1,
                                       m->chk, m->st);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpyAsync(m->hchk, m->chk, sizeof(int32_t), cudaMemcpyDeviceToHost, m->st));
        CUDA_TRY(cudaStreamSynchronize(m->st));
        if (*m->hchk < (int32_t)N) {
            sync_out(m);
            return fail(TRIME_EINVAL, "point " + std::to_string(*m->hchk) +
                                          " is not finite or outside the SDF grid box");
        }
    }
    if (cls) CUDA_TRY(cudaMemcpyAsync(scls, cls, N, cudaMemcpyHostToDevice, m->st));
    if (dprev) CUDA_TRY(cudaMemcpyAsync(sdp, dprev, N * sizeof(double), cudaMemcpyHostToDevice, m->st));
    if (m->prec == 0)
        launch_set_state<double>(make_args<double>(m, 1), p.soff, (int32_t)N, xy ? (const double*)sxy : nullptr,
                                 cls ? scls : nullptr, dprev ? sdp : nullptr, m->st);
    else
        launch_set_state<float>(make_args<float>(m, 1), p.soff, (int32_t)N, xy ? (const float*)sxy : nullptr,
                                cls ? scls : nullptr, dprev ? sdp : nullptr, m->st);
    CUDA_TRY(cudaGetLastError());
    if ((rc = force_retri(m, k))) return rc;
    CUDA_TRY(cudaStreamSynchronize(m->st));
    return sync_out(m);
}

static int get_state(mesh_s* m, int k, void* xy, uint8_t* cls, double* dprev) {
    const Part& p = m->parts[k];
    if (p.n == 0) return TRIME_OK;
    size_t N = (size_t)p.n, T = m->prec == 0 ? sizeof(double) : sizeof(float);
    int rc = sync_in(m);
    if (rc) return rc;
    // staging as in set_state: xy in xybuf, cls in tcnt, dprev in tbuf
    char* sxy = (char*)m->xybuf;
    uint8_t* scls = (uint8_t*)m->tcnt;
    double* sdp = (double*)m->tbuf;
    if (m->prec == 0)
        launch_get_state<double>(make_args<double>(m, 1), p.soff, (int32_t)N, xy ? (double*)sxy : nullptr,
                                 cls ? scls : nullptr, dprev ? sdp : nullptr, m->st);
    else
        launch_get_state<float>(make_args<float>(m, 1), p.soff, (int32_t)N, xy ? (float*)sxy : nullptr,
                                cls ? scls : nullptr, dprev ? sdp : nullptr, m->st);
    CUDA_TRY(cudaGetLastError());
    if (xy) CUDA_TRY(cudaMemcpyAsync(xy, sxy, 2 * N * T, cudaMemcpyDeviceToHost, m->st));
    if (cls) CUDA_TRY(cudaMemcpyAsync(cls, scls, N, cudaMemcpyDeviceToHost, m->st));
    if (dprev) CUDA_TRY(cudaMemcpyAsync(dprev, sdp, N * sizeof(double), cudaMemcpyDeviceToHost, m->st));
    CUDA_TRY(cudaStreamSynchronize(m->st));
    return sync_out(m);
}

static int set_method_state(mesh_s* m, int k, int32_t switched, double pa, double pb, double pm) {
    int rc = sync_in(m);
    if (rc) return rc;
    if ((rc = read_ctrl(m))) return rc;
    DevCtrl& c = m->hctrl[k];
    c.switched = switched;
    c.have_prev = pa > 0;
    c.prev_a = pa;
    c.prev_b = pb;
    c.prev_amax = pm;
    c.terminated = 0;
    c.small_moves = 0;
    c.retri = 1;
    CUDA_TRY(cudaMemcpyAsync(m->ctrl + k, &c, sizeof(DevCtrl), cudaMemcpyHostToDevice, m->st));
    CUDA_TRY(cudaStreamSynchronize(m->st));
    return sync_out(m);
}

template <typename T>
static int profile_stages(mesh_s* m, cudaEvent_t* ev) {
    IterArgs<T> a = make_args<T>(m, 0);
    CUDA_TRY(cudaEventRecord(ev[0], m->st));
    launch_bucket<T>(a, m->st);
    CUDA_TRY(cudaEventRecord(ev[1], m->st));
    launch_voronoi<T>(a, m->lanes, m->st);
    CUDA_TRY(cudaEventRecord(ev[2], m->st));
    launch_emit<T>(a, m->nblk, m->st);
    launch_dm_keep<T>(a, m->nblk, m->st);
    CUDA_TRY(cudaEventRecord(ev[3], m->st));
    launch_stats_pre<T>(a, 1, m->st);
    CUDA_TRY(cudaEventRecord(ev[4], m->st));
    launch_update<T>(a, m->nblk, m->st);
    CUDA_TRY(cudaEventRecord(ev[5], m->st));
    launch_stats_post<T>(a, m->st);
    CUDA_TRY(cudaEventRecord(ev[6], m->st));
    return 0;
}

static int profile(mesh_s* m, int32_t n_iters, double* stage_ms) {
    int rc = sync_in(m);
    if (rc) return rc;
    cudaEvent_t ev[7];
    for (int k = 0; k < 7; k++) CUDA_TRY(cudaEventCreate(&ev[k]));
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int32_t it = 0; it < n_iters && !rc; it++) {
        rc = m->prec == 0 ? profile_stages<double>(m, ev) : profile_stages<float>(m, ev);
        if (rc) break;
        CUDA_TRY(cudaEventSynchronize(ev[6]));
        for (int k = 0; k < 6; k++) {
            float ms = 0;
            CUDA_TRY(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
            acc[k] += ms;
        }
        float tot = 0;
        CUDA_TRY(cudaEventElapsedTime(&tot, ev[0], ev[6]));
        acc[6] += tot;
    }
    for (int k = 0; k < 7; k++) {
        stage_ms[k] += acc[k];
        cudaEventDestroy(ev[k]);
    }
    if (rc) return rc;
    CUDA_TRY(cudaGetLastError());
    return sync_out(m);
}

// new bucket size and Voronoi lane count: re-layout (growing the bucket
// arrays if needed) and capture the iteration again
static void drop_alloc(mesh_s* m, void* p) {
    auto it = std::find(m->allocs.begin(), m->allocs.end(), p);
    if (it != m->allocs.end()) m->allocs.erase(it);
    cudaFree(p);
}

static int set_tuning(mesh_s* m, double nopt, int32_t lanes) {
    if (!(nopt > 0) || (lanes != 8 && lanes != 16 && lanes != 32))
        return fail(TRIME_EINVAL, "n_opt must be > 0, lanes 8, 16 or 32");
    int rc = sync_in(m);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(m->st));
    if ((rc = layout_buckets(m, nopt))) return rc;
    if (m->nbtot > m->nbcap) {
        drop_alloc(m, m->bcount);
        drop_alloc(m, m->bstart);
        drop_alloc(m, m->scan_tmp);
        size_t scan_n = std::max<size_t>((size_t)m->nbtot + 1, (size_t)std::max(m->nslots, m->ncap) + 1);
        m->bcount = dalloc<int32_t>(m, (size_t)m->nbtot, rc);
        m->bstart = dalloc<int32_t>(m, (size_t)m->nbtot + 1, rc);
        m->scan_tmp = dalloc<int32_t>(m, scan_n / 4096 + 2, rc);
        if (rc) return rc;
        m->nbcap = m->nbtot;
    }
    m->lanes = lanes;
    if ((rc = upload_views(m)) || (rc = capture_graph(m))) return rc;
    return sync_out(m);
}

// ------------------------------------------------------------------ learned proposals (single mesh)
static int ensure_learn(mesh_s* m) {
    if (m->learn) return 0;
    size_t N = (size_t)std::max<int64_t>(m->nslots, 1), T = m->prec == 0 ? sizeof(double) : sizeof(float);
    LearnBufs* L = new LearnBufs();
    int rc = 0;
    L->X = dalloc<uint16_t>(m, N * kMlpIn, rc);
    L->Y = dalloc<float>(m, 2 * N, rc);
    L->H = dalloc<float>(m, N, rc);
    L->px = dalloc<char>(m, N * T, rc);
    L->py = dalloc<char>(m, N * T, rc);
    L->qx = dalloc<char>(m, N * T, rc);
    L->qy = dalloc<char>(m, N * T, rc);
    for (int b = 0; b < 2; b++) {
        L->bx[b] = dalloc<char>(m, N * T, rc);
        L->by[b] = dalloc<char>(m, N * T, rc);
        L->bdp[b] = dalloc<char>(m, N * T, rc);
        L->bid[b] = dalloc<int32_t>(m, N, rc);
        L->bcls[b] = dalloc<uint8_t>(m, N, rc);
    }
    if (rc) {
        delete L;
        return rc;
    }
    m->learn = L;
    return 0;
}

// the move of the next iteration is CVD
static float next_is_cvd(const mesh_s* m) {
    const DevCtrl& c = m->hctrl[0];
    return (c.method_param == 1 || (c.method_param == 2 && c.switched)) ? 1.0f : 0.0f;
}

// sort cur into srt at the current positions (a1) and compute the features;
// the last move is measured from the snapshot taken before the last iteration
template <typename T>
static void enqueue_features(mesh_s* m, uint16_t* X, float* H, void* px, void* py, int by_id, float mflag) {
    IterArgs<T> a = make_args<T>(m, 1);
    LearnBufs* L = m->learn;
    launch_bucket<T>(a, m->st);
    launch_features<T>(a, X, H, (T*)px, (T*)py, L->have_q ? (const T*)L->qx : nullptr,
                       L->have_q ? (const T*)L->qy : nullptr, by_id, mflag, m->st);
}

// remember the positions before the next iteration (the features' last move)
static void snapshot(mesh_s* m) {
    LearnBufs* L = m->learn;
    if (m->prec == 0) launch_snapshot<double>(make_args<double>(m, 1), (double*)L->qx, (double*)L->qy, m->st);
    else launch_snapshot<float>(make_args<float>(m, 1), (float*)L->qx, (float*)L->qy, m->st);
    L->have_q = true;
}

static void features_any(mesh_s* m, uint16_t* X, float* H, void* px, void* py, int by_id, float mflag) {
    if (m->prec == 0) enqueue_features<double>(m, X, H, px, py, by_id, mflag);
    else enqueue_features<float>(m, X, H, px, py, by_id, mflag);
    force_retri(m, -1);  // the sort above no longer matches the triangulation
    m->tri_stale = true;
}

static int check_net_err(mesh_s* m, mlp_s* net) {
    int h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, mlp_err(net), sizeof(int), cudaMemcpyDeviceToHost, m->st));
    CUDA_TRY(cudaStreamSynchronize(m->st));
    if (h) {
        cudaMemsetAsync(mlp_err(net), 0, sizeof(int), m->st);
        return fail(TRIME_ETIMEOUT, "tensor-core wait ran out");
    }
    return 0;
}

// features, network and proposed move on m's stream (the network's parameters
// are read from the model's memory; its own stream is not used)
static int enqueue_propose(mesh_s* m, mlp_s* net, double jump) {
    LearnBufs* L = m->learn;
    // a batch reads each mesh's move from its control block
    features_any(m, L->X, nullptr, nullptr, nullptr, 0, m->batched ? -1.0f : next_is_cvd(m));
    launch_mlp_forward(mlp_view(net), L->X, nullptr, (int)m->nslots, L->Y, mlp_err(net), m->st);
    if (m->prec == 0) launch_propose<double>(make_args<double>(m, 1), L->Y, (float)jump, m->st);
    else launch_propose<float>(make_args<float>(m, 1), L->Y, (float)jump, m->st);
    CUDA_TRY(cudaGetLastError());
    return 0;
}

static int copy_state(mesh_s* m, bool save, int b) {
    LearnBufs* L = m->learn;
    size_t N = (size_t)m->nslots, T = m->prec == 0 ? sizeof(double) : sizeof(float);
    auto cp = [&](void* cur, void* bak, size_t bytes) {
        return cudaMemcpyAsync(save ? bak : cur, save ? cur : bak, bytes, cudaMemcpyDeviceToDevice, m->st);
    };
    CUDA_TRY(cp(m->cx, L->bx[b], N * T));
    CUDA_TRY(cp(m->cy, L->by[b], N * T));
    CUDA_TRY(cp(m->cdp, L->bdp[b], N * T));
    CUDA_TRY(cp(m->cid, L->bid[b], N * sizeof(int32_t)));
    CUDA_TRY(cp(m->ccls, L->bcls[b], N));
    return 0;
}

static int write_ctrl0(mesh_s* m, const DevCtrl& c) {
    *m->hctrl = c;
    CUDA_TRY(cudaMemcpyAsync(m->ctrl, m->hctrl, sizeof(DevCtrl), cudaMemcpyHostToDevice, m->st));
    CUDA_TRY(cudaStreamSynchronize(m->st));
    return 0;
}

static int write_ctrl_all(mesh_s* m, const std::vector<DevCtrl>& c) {
    std::copy(c.begin(), c.end(), m->hctrl);
    CUDA_TRY(cudaMemcpyAsync(m->ctrl, m->hctrl, sizeof(DevCtrl) * c.size(), cudaMemcpyHostToDevice, m->st));
    CUDA_TRY(cudaStreamSynchronize(m->st));
    return 0;
}

// cur <- saved state b on the slots of the flagged parts (a single mesh is
// part 0; in a batch a slot's part is its chunk's)
template <typename T>
__global__ void k_restore_parts(int32_t n, const int32_t* cmesh, const uint8_t* flag, T* cx, T* cy, T* cdp,
                                int32_t* cid, uint8_t* ccls, const T* bx, const T* by, const T* bdp,
                                const int32_t* bid, const uint8_t* bcls) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n || !flag[cmesh ? cmesh[s >> kChunkShift] : 0]) return;
    cx[s] = bx[s];
    cy[s] = by[s];
    cdp[s] = bdp[s];
    cid[s] = bid[s];
    ccls[s] = bcls[s];
}

static int restore_parts(mesh_s* m, const std::vector<uint8_t>& flags, int b) {
    LearnBufs* L = m->learn;
    if (!L->rflag) {
        int rc = 0;
        L->rflag = dalloc<uint8_t>(m, flags.size(), rc);
        if (rc) return rc;
    }
    CUDA_TRY(cudaMemcpyAsync(L->rflag, flags.data(), flags.size(), cudaMemcpyHostToDevice, m->st));
    int n = (int)m->nslots, g = (n + kThreads - 1) / kThreads;
    const int32_t* cm = m->batched ? m->cmesh : nullptr;
    if (g > 0) {
        if (m->prec == 0)
            k_restore_parts<double><<<g, kThreads, 0, m->st>>>(n, cm, L->rflag, (double*)m->cx, (double*)m->cy,
                                                             (double*)m->cdp, m->cid, m->ccls, (double*)L->bx[b],
                                                             (double*)L->by[b], (double*)L->bdp[b], L->bid[b],
                                                             L->bcls[b]);
        else
            k_restore_parts<float><<<g, kThreads, 0, m->st>>>(n, cm, L->rflag, (float*)m->cx, (float*)m->cy,
                                                            (float*)m->cdp, m->cid, m->ccls, (float*)L->bx[b],
                                                            (float*)L->by[b], (float*)L->bdp[b], L->bid[b],
                                                            L->bcls[b]);
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(m->st));  // flags is the caller's host memory
    return 0;
}

// Learned proposals for a single mesh or every mesh of a batch: each
// proposal round runs, from the same state, one plain iteration and the
// proposal followed by one plain iteration; each mesh keeps the branch its
// own quality statistics favour (meshes that have terminated take no part).
static int do_step_learned(mesh_s* m, mlp_s* net, int32_t n_iters, int32_t every, double jump, double tol,
                           int32_t max_props, mesh_stats* stats, int32_t* accepted, int32_t* rejected) {
    int rc = sync_in(m);
    if (rc) return rc;
    if ((rc = ensure_learn(m)) || (rc = reset_counters(m)) || (rc = read_ctrl(m))) return rc;
    const size_t np = m->parts.size();
    std::vector<int> start(np), acc(np, 0), rej(np, 0);
    for (size_t p = 0; p < np; p++) start[p] = m->hctrl[p].iterations;
    int rounds = 0;
    if (n_iters > 0 && !all_terminated(m)) m->tri_stale = false;
    for (int32_t k = 0; k < n_iters && !all_terminated(m); k++) {
        if (k > 0 && k % every == 0 && m->nslots > 0 && (max_props <= 0 || rounds < max_props)) {
            // two branches from the same state: one plain iteration, and the
            // proposal followed by one plain iteration; the better one stays
            if ((rc = read_ctrl(m))) return rc;
            if (all_terminated(m)) break;
            const std::vector<DevCtrl> before(m->hctrl, m->hctrl + np);
            // plain branch (the last-move snapshot stays that of the saved state)
            if ((rc = copy_state(m, true, 0))) return rc;
            CUDA_TRY(cudaGraphLaunch(m->gexec, m->st));
            if ((rc = read_ctrl(m))) return rc;
            const std::vector<DevCtrl> plain(m->hctrl, m->hctrl + np);
            // proposal branch from the saved state
            if ((rc = copy_state(m, true, 1)) || (rc = copy_state(m, false, 0)) || (rc = force_retri(m, -1))) return rc;
            std::vector<DevCtrl> c0(before);
            for (size_t p = 0; p < np; p++) {
                c0[p].iterations = plain[p].iterations;
                c0[p].cnt = plain[p].cnt;
                c0[p].retri = 1;
            }
            if ((rc = write_ctrl_all(m, c0)) || (rc = enqueue_propose(m, net, jump))) return rc;
            snapshot(m);
            CUDA_TRY(cudaGraphLaunch(m->gexec, m->st));
            if ((rc = check_net_err(m, net)) || (rc = read_ctrl(m))) return rc;
            std::vector<DevCtrl> next(m->hctrl, m->hctrl + np);
            std::vector<uint8_t> lose(np, 0);
            bool any_lost = false;
            for (size_t p = 0; p < np; p++) {
                if (before[p].terminated) continue;
                const DevCtrl& after = next[p];
                // a proposal whose judged iteration tripped a capacity guard loses too
                bool guard = after.cnt.ring_overflow > plain[p].cnt.ring_overflow ||
                             after.cnt.exact_overflow > plain[p].cnt.exact_overflow;
                bool ok = !guard && after.n_tri > 0 && after.half_a < plain[p].half_a &&
                          after.min_ang >= plain[p].min_ang - tol;
                if (ok) {
                    acc[p]++;
                    continue;
                }
                rej[p]++;
                lose[p] = 1;
                any_lost = true;
                DevCtrl c = plain[p];
                c.iterations = after.iterations;
                c.cnt = after.cnt;
                c.cnt.ring_overflow = plain[p].cnt.ring_overflow;  // belonged to the discarded branch
                c.cnt.exact_overflow = plain[p].cnt.exact_overflow;
                c.cnt.clip_inconsistent = plain[p].cnt.clip_inconsistent;
                c.retri = 1;
                next[p] = c;
            }
            if (any_lost) {
                if ((rc = restore_parts(m, lose, 1)) || (rc = write_ctrl_all(m, next))) return rc;
                m->learn->have_q = false;  // the last move is unknown after the restore
            }
            rounds++;
            continue;
        }
        snapshot(m);
        CUDA_TRY(cudaGraphLaunch(m->gexec, m->st));
        if ((k & 31) == 31 && (rc = read_ctrl(m))) return rc;
    }
    if ((rc = read_ctrl(m)) || (rc = sync_out(m))) return rc;
    for (size_t p = 0; p < np; p++) {
        fill_stats(m, (int)p, m->hctrl[p].iterations - start[p], &stats[p]);
        if (accepted) accepted[p] = acc[p];
        if (rejected) rejected[p] = rej[p];
    }
    if (guard_tripped(m)) return TRIME_EDEVICE;
    return TRIME_OK;
}

// ------------------------------------------------------------------ C ABI
extern "C" {

void mesh_default_params(mesh_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->precision = 0;
    p->method = 2;
    p->bounded = 1;
    p->validity = 1;
    p->newton_max = 10;
    p->trace_max = 64;
    p->quad_max_level = 8;
    p->fac_F = 1.2;
    p->k_spring = 1.0;
    p->dt = 0.2;
    p->fac_pt = 0.4;
    p->fac_geps = 0.01;
    p->fac_voro_bound = 5.0;
    p->fac_end = 0.001;
    p->T_circ = 0.4;
    p->T_switch = 0.0015;
    p->T_end_q = 0.001;
    p->T_end_amax = 0.005;
    p->N_opt = 3.3;
    p->eta = 0.5;
    p->damping = 1.0;
    p->fac_retria = 0.1;
    p->fac_add = 0.6;
    p->T_add = 0.002;
    p->n_total = 0;
}

const char* mesh_last_error(void) { return g_err.c_str(); }

void mesh_destroy(mesh_t* m) {
    if (!m) return;
    destroy(m);
    delete m;
}

int mesh_init(mesh_t** out, const mesh_grid2d* sdf, const mesh_grid2d* sizing, const void* xy, int64_t n,
              const mesh_params* p, void* cuda_stream) {
    g_err.clear();
    if (!out) return fail(TRIME_EINVAL, "out is NULL");
    *out = nullptr;
    if (!sdf || !sizing) return fail(TRIME_EINVAL, "grid is NULL");
    mesh_params P;
    if (p) P = *p;
    else mesh_default_params(&P);
    mesh_s* m = new mesh_s();
    int rc = create(m, 1, sdf, sizing, &xy, &n, P, cuda_stream, 0);
    if (rc) {
        mesh_destroy(m);
        return rc;
    }
    *out = m;
    return TRIME_OK;
}

int mesh_rebuild(mesh_t* m, mesh_stats* stats) {
    if (!m) return fail(TRIME_EINVAL, "mesh is NULL");
    return do_rebuild(m, stats);
}

int mesh_step(mesh_t* m, int32_t n_iters, mesh_stats* stats) {
    if (!m) return fail(TRIME_EINVAL, "mesh is NULL");
    return do_step(m, n_iters, stats);
}

int mesh_get_state(mesh_t* m, void* xy, uint8_t* cls, double* dprev) {
    if (!m) return fail(TRIME_EINVAL, "mesh is NULL");
    return get_state(m, 0, xy, cls, dprev);
}

int mesh_init_points(const mesh_grid2d* sdf, const mesh_grid2d* sizing, int64_t n_init, uint64_t seed,
                     const mesh_params* p, double* xy, int64_t cap, int64_t* n_out, void* cuda_stream) {
    if (!sdf || !sizing || !n_out) return fail(TRIME_EINVAL, "NULL argument");
    if (n_init < 1 || n_init > (int64_t)1 << 30) return fail(TRIME_EINVAL, "n_init must be 1 .. 2^30");
    mesh_params P;
    if (p) P = *p;
    else mesh_default_params(&P);
    int rc = check_params(P);
    if (rc) return rc;
    if (!grid_ok(sdf) || !grid_ok(sizing)) return fail(TRIME_EINVAL, "invalid grid");
    for (size_t k = 0; k < (size_t)sizing->nx * sizing->ny; k++)
        if (!(sizing->v[k] > 0.0f)) return fail(TRIME_EINVAL, "sizing values must be positive");
    HostGeometry G;
    if ((rc = host_geometry(*sdf, *sizing, n_init, P, G))) return rc;
    // Sec. 3.5: Floyd-Steinberg dithering of n^E = rho_norm n_init over the
    // selected cells in row-major order, the residual passed in equal parts to
    // the selected neighbours not yet visited
    int ncx = sdf->nx - 1, ncy = sdf->ny - 1;
    size_t nc = (size_t)ncx * ncy;
    std::vector<double> carry(nc, 0.0);
    std::vector<int32_t> pcell;
    for (int gj = 0; gj < ncy; gj++)
        for (int gi = 0; gi < ncx; gi++) {
            size_t c = (size_t)gj * ncx + gi;
            if (!G.sel[c]) continue;
            double val = (G.rho[c] / G.sum_rho) * (double)n_init + carry[c];
            double k = std::floor(val + 0.5);
            if (k < 0.0) k = 0.0;
            double R = val - k;
            const int nb[4][2] = {{gi + 1, gj}, {gi - 1, gj + 1}, {gi, gj + 1}, {gi + 1, gj + 1}};
            int mn = 0;
            for (int q = 0; q < 4; q++)
                if (nb[q][0] >= 0 && nb[q][0] < ncx && nb[q][1] < ncy && G.sel[(size_t)nb[q][1] * ncx + nb[q][0]]) mn++;
            for (int q = 0; q < 4 && mn > 0; q++)
                if (nb[q][0] >= 0 && nb[q][0] < ncx && nb[q][1] < ncy && G.sel[(size_t)nb[q][1] * ncx + nb[q][0]])
                    carry[(size_t)nb[q][1] * ncx + nb[q][0]] += R / (double)mn;
            if ((int64_t)pcell.size() + (int64_t)k > (int64_t)1 << 30) return fail(TRIME_EINVAL, "too many points");
            pcell.insert(pcell.end(), (size_t)k, (int32_t)c);
        }
    int64_t n = (int64_t)pcell.size();
    *n_out = n;
    if (cap < n) return fail(TRIME_ECAPACITY, "point buffer too small");
    if (n == 0) return TRIME_OK;
    if (!xy) return fail(TRIME_EINVAL, "xy is NULL");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    size_t ns = (size_t)sdf->nx * sdf->ny;
    float* dsdf = nullptr;
    uint8_t* dcls = nullptr;
    double *dgeps = nullptr, *dout = nullptr;
    int32_t* dcell = nullptr;
    bool ok = cudaMalloc(&dsdf, ns * sizeof(float)) == cudaSuccess && cudaMalloc(&dcls, nc) == cudaSuccess &&
              cudaMalloc(&dgeps, nc * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&dout, 2 * (size_t)n * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&dcell, (size_t)n * sizeof(int32_t)) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(dsdf, sdf->v, ns * sizeof(float), cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(dcls, G.cls.data(), nc, cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(dgeps, G.geps.data(), nc * sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(dcell, pcell.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (ok) {
        launch_init_points(dev_grid(sdf, dsdf), dcls, dgeps, dcell, n, seed, P.damping, P.newton_max, dout, st);
        ok = cudaGetLastError() == cudaSuccess &&
             cudaMemcpyAsync(xy, dout, 2 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
             cudaStreamSynchronize(st) == cudaSuccess;
    }
    for (void* q : {(void*)dsdf, (void*)dcls, (void*)dgeps, (void*)dout, (void*)dcell})
        if (q) cudaFree(q);
    if (!ok) return fail(TRIME_ECUDA, "point initialisation on the device failed");
    return TRIME_OK;
}

int mesh_medial_points(mesh_t* m, double* v, uint8_t* flags) {
    if (!m || !v || !flags) return fail(TRIME_EINVAL, "NULL argument");
    const Part& p = m->parts[0];
    int rc = sync_in(m);
    if (rc) return rc;
    if (m->tri_stale) {
        enqueue(m, false, 1);
        if ((rc = force_retri(m, -1))) return rc;
        m->tri_stale = false;
    }
    if (p.n == 0) return sync_out(m);
    size_t n = (size_t)p.n;
    double* dv = nullptr;
    uint8_t* df = nullptr;
    CUDA_TRY(cudaMalloc(&dv, sizeof(double) * 4 * n));
    if (cudaMalloc(&df, n) != cudaSuccess) {
        cudaFree(dv);
        return fail(TRIME_ENOMEM, "cudaMalloc failed");
    }
    if (m->prec == 0) launch_medial<double>(make_args<double>(m, 1), (int32_t)p.n, dv, df, m->st);
    else launch_medial<float>(make_args<float>(m, 1), (int32_t)p.n, dv, df, m->st);
    // cells with more edges than a ring row: rebuilt by the big-cell pass
    int32_t nbig = 0;
    cudaError_t e = cudaMemcpyAsync(&nbig, m->ovf_n + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, m->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
    float4* scratch = nullptr;
    int32_t *rings = nullptr, *lens = nullptr;
    if (e == cudaSuccess && nbig > 0) {
        nbig = std::min<int32_t>(nbig, (int32_t)p.n);
        e = cudaMalloc(&scratch, sizeof(float4) * kBigScratchF4 * (size_t)nbig);
        if (e == cudaSuccess) e = cudaMalloc(&rings, sizeof(int32_t) * kBigRing * (size_t)nbig);
        if (e == cudaSuccess) e = cudaMalloc(&lens, sizeof(int32_t) * (size_t)nbig);
        if (e == cudaSuccess) {
            if (m->prec == 0) {
                launch_voronoi_big<double>(make_args<double>(m, 1), nbig, scratch, rings, lens, m->st);
                launch_medial_big<double>(make_args<double>(m, 1), nbig, rings, lens, dv, df, m->st);
            } else {
                launch_voronoi_big<float>(make_args<float>(m, 1), nbig, scratch, rings, lens, m->st);
                launch_medial_big<float>(make_args<float>(m, 1), nbig, rings, lens, dv, df, m->st);
            }
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(v, dv, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, m->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(flags, df, n, cudaMemcpyDeviceToHost, m->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
    cudaFree(dv);
    cudaFree(df);
    if (scratch) cudaFree(scratch);
    if (rings) cudaFree(rings);
    if (lens) cudaFree(lens);
    if (e != cudaSuccess) return fail(TRIME_ECUDA, std::string("medial points: ") + cudaGetErrorString(e));
    return sync_out(m);
}

int mesh_get_count(mesh_t* m, int64_t* n_current, int64_t* n_total) {
    if (!m) return fail(TRIME_EINVAL, "mesh is NULL");
    if (n_current) *n_current = m->parts[0].n;
    if (n_total) *n_total = m->ncap;
    return TRIME_OK;
}

int mesh_adf_cells(mesh_t* m, double fac_etol, int32_t* cells, double* tol, int64_t cap, int64_t* n_out) {
    if (!m || !n_out || (cap > 0 && (!cells || !tol))) return fail(TRIME_EINVAL, "NULL argument");
    if (m->batched) return fail(TRIME_EINVAL, "single meshes only");
    if (!(fac_etol >= 0.0) || !std::isfinite(fac_etol)) return fail(TRIME_EINVAL, "fac_etol must be finite, >= 0");
    const Part& p = m->parts[0];
    size_t nc = (size_t)(p.sdf.nx - 1) * (size_t)(p.sdf.ny - 1);
    std::vector<uint8_t> cls(nc);
    std::vector<double> geps(nc);
    int rc = sync_in(m);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(cls.data(), p.gcls, nc, cudaMemcpyDeviceToHost, m->st));
    CUDA_TRY(cudaMemcpyAsync(geps.data(), p.ggeps, nc * sizeof(double), cudaMemcpyDeviceToHost, m->st));
    CUDA_TRY(cudaStreamSynchronize(m->st));
    if ((rc = sync_out(m))) return rc;
    // Sec. 3.7: E_tol,i = fac_Etol geps_i fac_pt with fac_pt = sqrt(N_current / N_total)
    double fac_pt = std::sqrt((double)p.n / (double)std::max<int64_t>(m->ncap, 1));
    int64_t n = 0;
    for (size_t c = 0; c < nc; c++) {
        if (cls[c] != CELL_BOUNDARY) continue;
        if (n < cap) {
            cells[n] = (int32_t)c;
            tol[n] = fac_etol * geps[c] * fac_pt;
        }
        n++;
    }
    *n_out = n;
    if (n > cap) return fail(TRIME_ECAPACITY, "ADF cell buffers too small");
    return TRIME_OK;
}

int mesh_quality(mesh_t* m, mesh_quality_stats* q) {
    if (!m || !q) return fail(TRIME_EINVAL, "NULL argument");
    return quality(m, 0, q);
}

int mesh_get_triangles(mesh_t* m, int32_t* tri, int64_t cap, int64_t* n_out) {
    if (!m || !n_out) return fail(TRIME_EINVAL, "NULL argument");
    return get_triangles(m, 0, tri, cap, n_out);
}

int mesh_get_points(mesh_t* m, void* xy, int64_t cap, int64_t* n_out) {
    if (!m || !n_out) return fail(TRIME_EINVAL, "NULL argument");
    return get_points(m, 0, xy, cap, n_out);
}

int mesh_set_state(mesh_t* m, const void* xy, const uint8_t* cls, const double* dprev) {
    if (!m) return fail(TRIME_EINVAL, "mesh is NULL");
    return set_state(m, 0, xy, cls, dprev);
}

int mesh_set_method_state(mesh_t* m, int32_t switched, double pa, double pb, double pm) {
    if (!m) return fail(TRIME_EINVAL, "mesh is NULL");
    return set_method_state(m, 0, switched, pa, pb, pm);
}

int mesh_get_debug(mesh_t* m, int32_t what, double* out, int64_t cap) {
    if (!m || !out) return fail(TRIME_EINVAL, "NULL argument");
    if (!m->dbg) return fail(TRIME_EINVAL, "debug recording is off (mesh_params.debug = 1 enables it)");
    static const int off[7] = {0, 2, 4, 6, 7, 8, 9};
    static const int width[7] = {2, 2, 2, 1, 1, 1, 1};
    if (what < 0 || what > 6) return fail(TRIME_EINVAL, "what must be 0..6");
    int64_t n = m->nslots;
    size_t cnt = (size_t)width[what] * (size_t)n;
    if ((size_t)cap < cnt) return fail(TRIME_ECAPACITY, "debug buffer too small");
    if (cnt == 0) return TRIME_OK;
    int rc = sync_in(m);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(out, m->dbg + (size_t)off[what] * n, cnt * sizeof(double), cudaMemcpyDeviceToHost,
                             m->st));
    CUDA_TRY(cudaStreamSynchronize(m->st));
    return sync_out(m);
}

int mesh_profile_step(mesh_t* m, int32_t n_iters, double* stage_ms) {
    if (!m || !stage_ms || n_iters < 0) return fail(TRIME_EINVAL, "bad argument");
    return profile(m, n_iters, stage_ms);
}

static int set_target(mesh_s* m, int k, double min_angle) {
    int rc = sync_in(m);
    if (rc || (rc = read_ctrl(m))) return rc;
    size_t lo = k < 0 ? 0 : (size_t)k, hi = k < 0 ? m->parts.size() : (size_t)k + 1;
    for (size_t q = lo; q < hi; q++) {
        DevCtrl& c = m->hctrl[q];
        c.target_min_ang = min_angle;
        c.target_reached = 0;
        if (c.terminated && min_angle > 0 && !(c.min_ang >= min_angle)) c.terminated = 0;
        CUDA_TRY(cudaMemcpyAsync(m->ctrl + q, &c, sizeof(DevCtrl), cudaMemcpyHostToDevice, m->st));
    }
    CUDA_TRY(cudaStreamSynchronize(m->st));
    return sync_out(m);
}

int mesh_set_quality_target(mesh_t* m, double min_angle_deg) {
    if (!m || !(min_angle_deg >= 0) || min_angle_deg > 60) return fail(TRIME_EINVAL, "bad argument");
    return set_target(m, 0, min_angle_deg);
}

int mesh_set_tuning(mesh_t* m, double n_opt, int32_t lanes) {
    if (!m) return fail(TRIME_EINVAL, "mesh is NULL");
    return set_tuning(m, n_opt, lanes);
}

int mesh_features(mesh_t* m, uint16_t* X, float* h) {
    if (!m || !X) return fail(TRIME_EINVAL, "NULL argument");
    if (m->batched) return fail(TRIME_EINVAL, "single meshes only");
    if (growing(m)) return fail(TRIME_EINVAL, "learned proposals need N_current = N_total (point addition unfinished)");
    if (m->nslots == 0) return TRIME_OK;
    int rc = sync_in(m);
    if (rc || (rc = ensure_learn(m)) || (rc = read_ctrl(m))) return rc;
    size_t N = (size_t)m->nslots;
    bool dx = is_device_ptr(X), dh = h && is_device_ptr(h);
    features_any(m, dx ? X : m->learn->X, h ? (dh ? h : m->learn->H) : nullptr, nullptr, nullptr, 1, next_is_cvd(m));
    CUDA_TRY(cudaGetLastError());
    if (!dx) CUDA_TRY(cudaMemcpyAsync(X, m->learn->X, N * kMlpIn * 2, cudaMemcpyDeviceToHost, m->st));
    if (h && !dh) CUDA_TRY(cudaMemcpyAsync(h, m->learn->H, N * sizeof(float), cudaMemcpyDeviceToHost, m->st));
    CUDA_TRY(cudaStreamSynchronize(m->st));
    return sync_out(m);
}

int mesh_collect_pairs(mesh_t* m, int32_t horizon, uint16_t* X, float* T) {
    if (!m || !X || !T || horizon < 1) return fail(TRIME_EINVAL, "bad argument");
    if (m->batched) return fail(TRIME_EINVAL, "single meshes only");
    if (growing(m)) return fail(TRIME_EINVAL, "learned proposals need N_current = N_total (point addition unfinished)");
    if (!is_device_ptr(X) || !is_device_ptr(T)) return fail(TRIME_EINVAL, "X and T must be device arrays");
    if (m->nslots == 0) return TRIME_OK;
    int rc = sync_in(m);
    if (rc || (rc = ensure_learn(m)) || (rc = read_ctrl(m))) return rc;
    LearnBufs* L = m->learn;
    snapshot(m);
    CUDA_TRY(cudaGraphLaunch(m->gexec, m->st));
    if ((rc = read_ctrl(m))) return rc;
    features_any(m, X, L->H, L->px, L->py, 1, next_is_cvd(m));
    for (int32_t k = 0; k < horizon; k++) CUDA_TRY(cudaGraphLaunch(m->gexec, m->st));
    if (m->prec == 0)
        launch_targets<double>(make_args<double>(m, 1), (const double*)L->px, (const double*)L->py, L->H, T, m->st);
    else
        launch_targets<float>(make_args<float>(m, 1), (const float*)L->px, (const float*)L->py, L->H, T, m->st);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(m->st));
    return sync_out(m);
}

int mesh_propose(mesh_t* m, mlp_t* net, double jump) {
    if (!m || !net || !(jump > 0)) return fail(TRIME_EINVAL, "bad argument");
    if (m->batched) return fail(TRIME_EINVAL, "single meshes only");
    if (growing(m)) return fail(TRIME_EINVAL, "learned proposals need N_current = N_total (point addition unfinished)");
    if (m->nslots == 0) return TRIME_OK;
    int rc = sync_in(m);
    if (rc || (rc = ensure_learn(m)) || (rc = read_ctrl(m)) || (rc = enqueue_propose(m, net, jump))) return rc;
    if ((rc = check_net_err(m, net))) return rc;
    return sync_out(m);
}

int mesh_step_learned(mesh_t* m, mlp_t* net, int32_t n_iters, int32_t every, double jump, double min_angle_tol,
                      int32_t max_proposals, mesh_stats* stats, int32_t* accepted, int32_t* rejected) {
    if (!m || !net || !stats || n_iters < 0 || every < 1 || !(jump > 0) || !(min_angle_tol >= 0))
        return fail(TRIME_EINVAL, "bad argument");
    if (m->batched) return fail(TRIME_EINVAL, "single meshes only");
    if (growing(m)) return fail(TRIME_EINVAL, "learned proposals need N_current = N_total (point addition unfinished)");
    return do_step_learned(m, net, n_iters, every, jump, min_angle_tol, max_proposals, stats, accepted, rejected);
}

// ------------------------------------------------------------------ batches
int mesh_batch_init(mesh_batch_t** out, int32_t n_meshes, const mesh_grid2d* sdfs, const mesh_grid2d* sizings,
                    const void* const* xys, const int64_t* ns, const mesh_params* p, int32_t autotune,
                    void* cuda_stream) {
    g_err.clear();
    if (!out) return fail(TRIME_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_meshes < 1 || n_meshes > (1 << 20)) return fail(TRIME_EINVAL, "n_meshes out of range");
    if (!sdfs || !sizings || !xys || !ns) return fail(TRIME_EINVAL, "NULL array");
    mesh_params P;
    if (p) P = *p;
    else mesh_default_params(&P);
    mesh_batch_s* b = new mesh_batch_s();
    b->batched = true;
    int rc = create(b, n_meshes, sdfs, sizings, xys, ns, P, cuda_stream, autotune != 0);
    if (rc) {
        mesh_batch_destroy(b);
        return rc;
    }
    *out = b;
    return TRIME_OK;
}

void mesh_batch_destroy(mesh_batch_t* b) {
    if (!b) return;
    destroy(b);
    delete b;
}

int mesh_batch_size(const mesh_batch_t* b) { return b ? (int)b->parts.size() : 0; }

int mesh_batch_rebuild(mesh_batch_t* b, mesh_stats* stats) {
    if (!b) return fail(TRIME_EINVAL, "batch is NULL");
    return do_rebuild(b, stats);
}

int mesh_batch_step(mesh_batch_t* b, int32_t n_iters, mesh_stats* stats) {
    if (!b) return fail(TRIME_EINVAL, "batch is NULL");
    return do_step(b, n_iters, stats);
}

static int check_mesh(const mesh_batch_t* b, int32_t mesh) {
    if (!b) return fail(TRIME_EINVAL, "batch is NULL");
    if (mesh < 0 || mesh >= (int32_t)b->parts.size()) return fail(TRIME_EINVAL, "mesh index out of range");
    return 0;
}

int mesh_batch_get_triangles(mesh_batch_t* b, int32_t mesh, int32_t* tri, int64_t cap, int64_t* n_out) {
    int rc = check_mesh(b, mesh);
    if (rc) return rc;
    if (!n_out) return fail(TRIME_EINVAL, "n_out is NULL");
    return get_triangles(b, mesh, tri, cap, n_out);
}

int mesh_batch_get_points(mesh_batch_t* b, int32_t mesh, void* xy, int64_t cap, int64_t* n_out) {
    int rc = check_mesh(b, mesh);
    if (rc) return rc;
    if (!n_out) return fail(TRIME_EINVAL, "n_out is NULL");
    return get_points(b, mesh, xy, cap, n_out);
}

int mesh_batch_set_state(mesh_batch_t* b, int32_t mesh, const void* xy, const uint8_t* cls, const double* dprev) {
    int rc = check_mesh(b, mesh);
    if (rc) return rc;
    return set_state(b, mesh, xy, cls, dprev);
}

int mesh_batch_set_method_state(mesh_batch_t* b, int32_t mesh, int32_t switched, double pa, double pb, double pm) {
    int rc = check_mesh(b, mesh);
    if (rc) return rc;
    return set_method_state(b, mesh, switched, pa, pb, pm);
}

int mesh_batch_profile_step(mesh_batch_t* b, int32_t n_iters, double* stage_ms) {
    if (!b || !stage_ms || n_iters < 0) return fail(TRIME_EINVAL, "bad argument");
    return profile(b, n_iters, stage_ms);
}

int mesh_batch_set_quality_target(mesh_batch_t* b, int32_t mesh, double min_angle_deg) {
    if (!b || !(min_angle_deg >= 0) || min_angle_deg > 60) return fail(TRIME_EINVAL, "bad argument");
    if (mesh < -1 || mesh >= (int32_t)b->parts.size()) return fail(TRIME_EINVAL, "mesh index out of range");
    return set_target(b, mesh, min_angle_deg);
}

int mesh_batch_quality(mesh_batch_t* b, int32_t mesh, mesh_quality_stats* q) {
    if (!b || !q) return fail(TRIME_EINVAL, "NULL argument");
    if (mesh < 0 || mesh >= (int32_t)b->parts.size()) return fail(TRIME_EINVAL, "mesh index out of range");
    return quality(b, mesh, q);
}

int mesh_batch_step_learned(mesh_batch_t* b, mlp_t* net, int32_t n_iters, int32_t every, double jump,
                            double min_angle_tol, int32_t max_rounds, mesh_stats* stats, int32_t* accepted,
                            int32_t* rejected) {
    if (!b || !net || !stats || n_iters < 0 || every < 1 || !(jump > 0) || !(min_angle_tol >= 0))
        return fail(TRIME_EINVAL, "bad argument");
    return do_step_learned(b, net, n_iters, every, jump, min_angle_tol, max_rounds, stats, accepted, rejected);
}

int mesh_batch_set_tuning(mesh_batch_t* b, double n_opt, int32_t lanes) {
    if (!b) return fail(TRIME_EINVAL, "batch is NULL");
    return set_tuning(b, n_opt, lanes);
}

int mesh_batch_get_tuning(const mesh_batch_t* b, mesh_tuning* out) {
    if (!b || !out) return fail(TRIME_EINVAL, "NULL argument");
    std::memset(out, 0, sizeof *out);
    out->n_opt = b->nopt;
    out->lanes = b->lanes;
    out->n_slots = b->nslots;
    out->n_buckets = b->nbtot;
    int nc = (int)std::min<size_t>(b->tune.size(), 12);
    out->n_candidates = nc;
    for (int k = 0; k < nc; k++) {
        out->cand_n_opt[k] = b->tune[k].nopt;
        out->cand_lanes[k] = b->tune[k].lanes;
        out->cand_ms[k] = b->tune[k].ms;
    }
    return TRIME_OK;
}

int mesh_bucket_points(const double* x, const double* y, int64_t n, double x0, double y0, double x1, double y1,
                       int32_t nbx, int32_t nby, int32_t* bucket_start, int32_t* sorted_idx, int32_t* scratch,
                       void* cuda_stream) {
    if (n < 0 || n > (int64_t)(1 << 30)) return fail(TRIME_EINVAL, "n out of range");
    if (nbx < 1 || nby < 1 || (int64_t)nbx * nby > (int64_t)4096 * 1024) return fail(TRIME_EINVAL, "bad bucket grid");
    if (!(x1 > x0) || !(y1 > y0)) return fail(TRIME_EINVAL, "empty box");
    if (!bucket_start || !scratch || (n > 0 && (!x || !y || !sorted_idx))) return fail(TRIME_EINVAL, "NULL pointer");
    launch_bucket_raw(x, y, (int32_t)n, x0, y0, (x1 - x0) / nbx, (y1 - y0) / nby, nbx, nby, bucket_start, sorted_idx,
                      scratch, (cudaStream_t)cuda_stream);
    CUDA_TRY(cudaGetLastError());
    return TRIME_OK;
}

int mesh_exact_predicates(const double* pts, const int32_t* ids, int64_t nq, int32_t* out_orient,
                          int32_t* out_incircle) {
    if (nq < 0 || nq > (int64_t)(1 << 26)) return fail(TRIME_EINVAL, "nq out of range");
    if (nq == 0) return TRIME_OK;
    if (!pts || !ids || !out_orient || !out_incircle) return fail(TRIME_EINVAL, "NULL pointer");
    double* dp = nullptr;
    int32_t *di = nullptr, *dout = nullptr;
    size_t n = (size_t)nq;
    if (cudaMalloc(&dp, 8 * n * sizeof(double)) != cudaSuccess || cudaMalloc(&di, 4 * n * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&dout, 2 * n * sizeof(int32_t)) != cudaSuccess) {
        cudaFree(dp);
        cudaFree(di);
        cudaFree(dout);
        return fail(TRIME_ENOMEM, "cudaMalloc failed");
    }
    cudaError_t e = cudaMemcpy(dp, pts, 8 * n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(di, ids, 4 * n * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        launch_predicates(dp, di, (int32_t)nq, dout, dout + n, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out_orient, dout, n * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out_incircle, dout + n, n * sizeof(int32_t), cudaMemcpyDeviceToHost);
    cudaFree(dp);
    cudaFree(di);
    cudaFree(dout);
    if (e != cudaSuccess) return fail(TRIME_ECUDA, std::string("predicates: ") + cudaGetErrorString(e));
    return TRIME_OK;
}

}  // extern "C"
