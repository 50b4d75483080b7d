/*
 * trime_oracle.c -- plain FP64 CPU oracle for one TriMe++ meshing iteration.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
 * CPU baseline of bench.py; never by the product path.  Shares no code with
 * the CUDA library.  Compile with -O2 -ffp-contract=off and no fast-math: the
 * fixed floating-point formulas below are part of the triangle-set definition.
 *
 * Paper: TriMe++ (Lu & Rycroft, arXiv 2309.13824).  Section numbers refer to it.
 */
#include "trime_oracle.h"

#include <math.h>
#include <omp.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* error reporting                                                          */
/* ------------------------------------------------------------------------ */
static char g_err[256];
static void set_err(const char* s) { snprintf(g_err, sizeof g_err, "%s", s); }
const char* om_last_error(void) { return g_err; }

/* ------------------------------------------------------------------------ */
/* Exact arithmetic: sign-magnitude big integers, base 2^32.                */
/* Every double is m * 2^e with integer m < 2^53; a predicate scales all its */
/* inputs by 2^-emin so they become integers and evaluates its determinant  */
/* exactly.  Capacity covers degree-4 products over the full double range.  */
/* ------------------------------------------------------------------------ */
#define BI_MAX 352
typedef struct {
    int neg;
    int n;
    uint32_t d[BI_MAX];
} bi_t;

static void bi_norm(bi_t* a) {
    while (a->n > 0 && a->d[a->n - 1] == 0) a->n--;
    if (a->n == 0) a->neg = 0;
}

static int bi_cmp_mag(const bi_t* a, const bi_t* b) {
    if (a->n != b->n) return a->n < b->n ? -1 : 1;
    for (int k = a->n - 1; k >= 0; k--)
        if (a->d[k] != b->d[k]) return a->d[k] < b->d[k] ? -1 : 1;
    return 0;
}

/* r = |a| + |b| (r may alias) */
static void bi_add_mag(bi_t* r, const bi_t* a, const bi_t* b) {
    int n = a->n > b->n ? a->n : b->n;
    uint64_t carry = 0;
    for (int k = 0; k < n; k++) {
        uint64_t s = carry;
        if (k < a->n) s += a->d[k];
        if (k < b->n) s += b->d[k];
        r->d[k] = (uint32_t)s;
        carry = s >> 32;
    }
    if (carry) {
        if (n >= BI_MAX) { fprintf(stderr, "oracle bigint overflow\n"); abort(); }
        r->d[n++] = (uint32_t)carry;
    }
    r->n = n;
}

/* r = |a| - |b|, requires |a| >= |b| (r may alias) */
static void bi_sub_mag(bi_t* r, const bi_t* a, const bi_t* b) {
    int64_t borrow = 0;
    for (int k = 0; k < a->n; k++) {
        int64_t s = (int64_t)a->d[k] - borrow - (k < b->n ? (int64_t)b->d[k] : 0);
        if (s < 0) { s += ((int64_t)1 << 32); borrow = 1; } else borrow = 0;
        r->d[k] = (uint32_t)s;
    }
    r->n = a->n;
}

/* r = a + b (signed; r may alias a or b) */
static void bi_add(bi_t* r, const bi_t* a, const bi_t* b) {
    if (a->neg == b->neg) {
        int neg = a->neg;
        bi_add_mag(r, a, b);
        r->neg = neg;
    } else {
        int c = bi_cmp_mag(a, b);
        if (c == 0) { r->n = 0; r->neg = 0; return; }
        if (c > 0) { int neg = a->neg; bi_sub_mag(r, a, b); r->neg = neg; }
        else { int neg = b->neg; bi_sub_mag(r, b, a); r->neg = neg; }
    }
    bi_norm(r);
}

static void bi_sub(bi_t* r, const bi_t* a, const bi_t* b) {
    bi_t nb = *b;
    if (nb.n) nb.neg = !nb.neg;
    bi_add(r, a, &nb);
}

static void bi_mul(bi_t* r, const bi_t* a, const bi_t* b) {
    bi_t t;
    if (a->n == 0 || b->n == 0) { r->n = 0; r->neg = 0; return; }
    int n = a->n + b->n;
    if (n > BI_MAX) { fprintf(stderr, "oracle bigint overflow\n"); abort(); }
    memset(t.d, 0, sizeof(uint32_t) * (size_t)n);
    for (int i = 0; i < a->n; i++) {
        uint64_t carry = 0;
        for (int j = 0; j < b->n; j++) {
            uint64_t cur = (uint64_t)a->d[i] * b->d[j] + t.d[i + j] + carry;
            t.d[i + j] = (uint32_t)cur;
            carry = cur >> 32;
        }
        int k = i + b->n;
        while (carry) {
            uint64_t cur = (uint64_t)t.d[k] + carry;
            t.d[k] = (uint32_t)cur;
            carry = cur >> 32;
            k++;
        }
    }
    t.n = n;
    t.neg = a->neg ^ b->neg;
    bi_norm(&t);
    *r = t;
}

static int bi_sign(const bi_t* a) { return a->n == 0 ? 0 : (a->neg ? -1 : 1); }

/* x = +-M * 2^e with M < 2^53 an integer */
static void dbl_split(double x, uint64_t* M, int* e, int* neg) {
    if (x == 0.0) { *M = 0; *e = 0; *neg = 0; return; }
    int E;
    double f = frexp(fabs(x), &E);
    *M = (uint64_t)ldexp(f, 53);
    *e = E - 53;
    *neg = x < 0;
}

/* Convert n doubles to integers sharing the scale 2^emin. */
static void bi_from_doubles(const double* x, int n, bi_t* out) {
    uint64_t M[8];
    int e[8], neg[8];
    int emin = 1 << 30;
    for (int k = 0; k < n; k++) {
        dbl_split(x[k], &M[k], &e[k], &neg[k]);
        if (M[k] && e[k] < emin) emin = e[k];
    }
    for (int k = 0; k < n; k++) {
        bi_t* r = &out[k];
        r->neg = 0;
        r->n = 0;
        if (!M[k]) continue;
        int sh = e[k] - emin;
        int w = sh / 32, b = sh % 32;
        int top = w + 3;
        if (top > BI_MAX) { fprintf(stderr, "oracle bigint overflow\n"); abort(); }
        memset(r->d, 0, sizeof(uint32_t) * (size_t)top);
        /* place M << b at word w */
        unsigned __int128 v = (unsigned __int128)M[k] << b;
        r->d[w] = (uint32_t)v;
        r->d[w + 1] = (uint32_t)(v >> 32);
        r->d[w + 2] = (uint32_t)(v >> 64);
        r->n = top;
        r->neg = neg[k];
        bi_norm(r);
    }
}

/* ------------------------------------------------------------------------ */
/* Exact predicates.  orient2d(a,b,c) = (b-a) x (c-a) > 0 for CCW.           */
/* incircle(a,b,c,d) = det of rows [x, y, x^2+y^2, 1]; > 0 iff d inside the  */
/* circle through CCW a,b,c.  A loose double filter decides easy cases.     */
/* ------------------------------------------------------------------------ */
static int orient_exact_bi(const double* a, const double* b, const double* c) {
    double in[6] = {a[0], a[1], b[0], b[1], c[0], c[1]};
    bi_t X[6], t1, t2, u, v;
    bi_from_doubles(in, 6, X);
    bi_sub(&t1, &X[2], &X[0]); /* bx-ax */
    bi_sub(&t2, &X[5], &X[1]); /* cy-ay */
    bi_mul(&u, &t1, &t2);
    bi_sub(&t1, &X[3], &X[1]); /* by-ay */
    bi_sub(&t2, &X[4], &X[0]); /* cx-ax */
    bi_mul(&v, &t1, &t2);
    bi_sub(&u, &u, &v);
    return bi_sign(&u);
}

int om_orient2d(const double* a, const double* b, const double* c) {
    double l = (b[0] - a[0]) * (c[1] - a[1]);
    double r = (b[1] - a[1]) * (c[0] - a[0]);
    double det = l - r, sum = fabs(l) + fabs(r);
    if (isfinite(det) && isfinite(sum) && sum > 1e-200 && fabs(det) > 1e-12 * sum)
        return det > 0 ? 1 : -1;
    return orient_exact_bi(a, b, c);
}

static int incircle_exact_bi(const double* a, const double* b, const double* c, const double* d) {
    double in[8] = {a[0], a[1], b[0], b[1], c[0], c[1], d[0], d[1]};
    bi_t X[8], adx, ady, bdx, bdy, cdx, cdy, al, bl, cl, t, u, det;
    bi_from_doubles(in, 8, X);
    bi_sub(&adx, &X[0], &X[6]); bi_sub(&ady, &X[1], &X[7]);
    bi_sub(&bdx, &X[2], &X[6]); bi_sub(&bdy, &X[3], &X[7]);
    bi_sub(&cdx, &X[4], &X[6]); bi_sub(&cdy, &X[5], &X[7]);
    bi_mul(&t, &adx, &adx); bi_mul(&u, &ady, &ady); bi_add(&al, &t, &u);
    bi_mul(&t, &bdx, &bdx); bi_mul(&u, &bdy, &bdy); bi_add(&bl, &t, &u);
    bi_mul(&t, &cdx, &cdx); bi_mul(&u, &cdy, &cdy); bi_add(&cl, &t, &u);
    /* al*(bdx*cdy - bdy*cdx) */
    bi_mul(&t, &bdx, &cdy); bi_mul(&u, &bdy, &cdx); bi_sub(&t, &t, &u); bi_mul(&det, &al, &t);
    /* + bl*(cdx*ady - cdy*adx) */
    bi_mul(&t, &cdx, &ady); bi_mul(&u, &cdy, &adx); bi_sub(&t, &t, &u); bi_mul(&t, &bl, &t);
    bi_add(&det, &det, &t);
    /* + cl*(adx*bdy - ady*bdx) */
    bi_mul(&t, &adx, &bdy); bi_mul(&u, &ady, &bdx); bi_sub(&t, &t, &u); bi_mul(&t, &cl, &t);
    bi_add(&det, &det, &t);
    return bi_sign(&det);
}

int om_incircle(const double* a, const double* b, const double* c, const double* d) {
    double adx = a[0] - d[0], ady = a[1] - d[1];
    double bdx = b[0] - d[0], bdy = b[1] - d[1];
    double cdx = c[0] - d[0], cdy = c[1] - d[1];
    double al = adx * adx + ady * ady, bl = bdx * bdx + bdy * bdy, cl = cdx * cdx + cdy * cdy;
    double m1 = bdx * cdy - bdy * cdx, m2 = cdx * ady - cdy * adx, m3 = adx * bdy - ady * bdx;
    double det = al * m1 + bl * m2 + cl * m3;
    double perm = al * (fabs(bdx * cdy) + fabs(bdy * cdx)) + bl * (fabs(cdx * ady) + fabs(cdy * adx)) +
                  cl * (fabs(adx * bdy) + fabs(ady * bdx));
    if (isfinite(det) && isfinite(perm) && perm > 1e-150 && fabs(det) > 1e-11 * perm)
        return det > 0 ? 1 : -1;
    return incircle_exact_bi(a, b, c, d);
}

/* Symbolic perturbation: the lifted coordinate of point r becomes
 * |p_r|^2 + eps^(id_r + 1), so smaller ids carry larger perturbations.  The
 * perturbed det4 is det4 + sum_r eps_r C_r with C_a = orient(b,c,d),
 * C_b = -orient(a,c,d), C_c = orient(a,b,d), C_d = -orient(a,b,c). */
int om_incircle_sos(const double* a, int64_t ia, const double* b, int64_t ib,
                    const double* c, int64_t ic, const double* d, int64_t id) {
    int s = om_incircle(a, b, c, d);
    if (s) return s;
    const double* P[4] = {a, b, c, d};
    int64_t I[4] = {ia, ib, ic, id};
    int ord[4] = {0, 1, 2, 3};
    for (int i = 1; i < 4; i++)
        for (int j = i; j > 0 && I[ord[j]] < I[ord[j - 1]]; j--) {
            int t = ord[j]; ord[j] = ord[j - 1]; ord[j - 1] = t;
        }
    for (int q = 0; q < 4; q++) {
        int r = ord[q];
        int cs;
        switch (r) {
            case 0: cs = om_orient2d(P[1], P[2], P[3]); break;
            case 1: cs = -om_orient2d(P[0], P[2], P[3]); break;
            case 2: cs = om_orient2d(P[0], P[1], P[3]); break;
            default: cs = -om_orient2d(P[0], P[1], P[2]); break;
        }
        if (cs) return cs;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Grids and the fixed bilinear formula                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nx, ny;
    double x0, y0, x1, y1, dx, dy;
    float* v;
} grid_t;

static int grid_copy(grid_t* g, const om_grid* s) {
    if (!s || s->nx < 2 || s->ny < 2 || !s->v || !(s->x1 > s->x0) || !(s->y1 > s->y0)) return -1;
    g->nx = s->nx; g->ny = s->ny;
    g->x0 = s->x0; g->y0 = s->y0; g->x1 = s->x1; g->y1 = s->y1;
    g->dx = (s->x1 - s->x0) / (double)(s->nx - 1);
    g->dy = (s->y1 - s->y0) / (double)(s->ny - 1);
    size_t n = (size_t)s->nx * (size_t)s->ny;
    g->v = (float*)malloc(n * sizeof(float));
    if (!g->v) return -1;
    memcpy(g->v, s->v, n * sizeof(float));
    for (size_t k = 0; k < n; k++)
        if (!isfinite(g->v[k])) return -1;
    return 0;
}

/* cell and local coordinates, clamped to the grid */
static void grid_locate(const grid_t* g, double x, double y, int* i, int* j, double* fx, double* fy) {
    double tx = (x - g->x0) / g->dx, ty = (y - g->y0) / g->dy;
    double fi = floor(tx), fj = floor(ty);
    int ii, jj;
    if (!(fi >= 0.0)) ii = 0; else if (fi > (double)(g->nx - 2)) ii = g->nx - 2; else ii = (int)fi;
    if (!(fj >= 0.0)) jj = 0; else if (fj > (double)(g->ny - 2)) jj = g->ny - 2; else jj = (int)fj;
    double ax = tx - (double)ii, ay = ty - (double)jj;
    if (ax < 0.0) ax = 0.0; if (ax > 1.0) ax = 1.0;
    if (ay < 0.0) ay = 0.0; if (ay > 1.0) ay = 1.0;
    *i = ii; *j = jj; *fx = ax; *fy = ay;
}

static double bilin(const grid_t* g, double x, double y) {
    int i, j;
    double fx, fy;
    grid_locate(g, x, y, &i, &j, &fx, &fy);
    const float* r0 = g->v + (size_t)j * g->nx + i;
    const float* r1 = r0 + g->nx;
    double v00 = r0[0], v10 = r0[1], v01 = r1[0], v11 = r1[1];
    double a = v00 + fx * (v10 - v00);
    double b = v01 + fx * (v11 - v01);
    return a + fy * (b - a);
}

/* exact derivatives of the bilinear interpolant (f_xx = f_yy = 0) */
static void bilin_d(const grid_t* g, double x, double y, double* f, double* fx_, double* fy_, double* fxy) {
    int i, j;
    double fx, fy;
    grid_locate(g, x, y, &i, &j, &fx, &fy);
    const float* r0 = g->v + (size_t)j * g->nx + i;
    const float* r1 = r0 + g->nx;
    double v00 = r0[0], v10 = r0[1], v01 = r1[0], v11 = r1[1];
    double a = v00 + fx * (v10 - v00);
    double b = v01 + fx * (v11 - v01);
    *f = a + fy * (b - a);
    double d0 = v10 - v00, d1 = v11 - v01;
    *fx_ = (d0 + fy * (d1 - d0)) / g->dx;
    *fy_ = (b - a) / g->dy;
    *fxy = (d1 - d0) / (g->dx * g->dy);
}

double om_bilinear(const om_grid* s, double x, double y) {
    grid_t g;
    g.nx = s->nx; g.ny = s->ny; g.x0 = s->x0; g.y0 = s->y0; g.x1 = s->x1; g.y1 = s->y1;
    g.dx = (s->x1 - s->x0) / (double)(s->nx - 1);
    g.dy = (s->y1 - s->y0) / (double)(s->ny - 1);
    g.v = (float*)s->v;
    return bilin(&g, x, y);
}

/* ------------------------------------------------------------------------ */
/* Mesh state                                                               */
/* ------------------------------------------------------------------------ */
enum { CLS_INNER = 0, CLS_BOUNDARY = 1, CLS_OUTER = 2 };
enum { PT_INNER = 0, PT_BOUNDARY = 1, PT_OUTSIDE = 2 };

typedef struct { double nx, ny, s; int32_t lab; } hp_t; /* n.u <= s, u relative to the generator */

#define CELL_CAP 512

struct om_mesh {
    om_params P;
    int64_t N;                 /* N_current */
    int64_t Ntot;              /* N_total (>= N; arrays hold Ntot points) */
    double *x, *y;
    uint8_t* cls;
    double* dprev;
    grid_t sdf, siz;
    int ncx, ncy;
    double ldiag, havg;
    uint8_t* gcls;
    double *gh, *ggeps;
    /* rebuild products */
    int64_t* ring_off;
    int32_t* ring;
    int64_t ring_cap;
    int64_t ntri;
    int32_t* tri;
    int64_t nedge;
    int32_t* edge;
    /* step products */
    double *pnew, *force, *fsum, *cen, *area;
    int32_t* qlevel;
    om_stats st;
    int retri;                 /* the next step re-triangulates (Algorithm 1) */
    double *tx, *ty;           /* positions at the last triangulation */
    int switched, have_prev;
    double prev_a, prev_b, prev_amax;
    int64_t clip_errors;
    int threads;               /* OpenMP threads of the per-cell loops (results do not depend on it) */
};

void om_default_params(om_params* p) {
    memset(p, 0, sizeof *p);
    p->method = 2;
    p->bounded = 1;
    p->validity = 1;
    p->newton_max = 10;       /* App. B: T_ct^newton */
    p->trace_max = 64;
    p->quad_max_level = 8;
    p->fac_F = 1.2;           /* App. B */
    p->k_spring = 1.0;
    p->dt = 0.2;
    p->fac_pt = 0.4;          /* App. B: fac_mvmt^pt */
    p->fac_geps = 0.01;       /* App. B */
    p->fac_voro_bound = 5.0;  /* App. B */
    p->fac_end = 0.001;       /* App. B: fac_mvmt^end */
    p->T_circ = 0.4;          /* App. B */
    p->T_switch = 0.0015;     /* App. B */
    p->T_end_q = 0.001;       /* App. B */
    p->T_end_amax = 0.005;    /* App. B */
    p->N_opt = 3.3;           /* App. B */
    p->eta = 0.5;             /* App. B */
    p->damping = 1.0;         /* App. B: alpha-hat */
    p->fac_retria = 0.1;      /* App. B: fac_mvmt^retria (DistMesh only) */
    p->fac_add = 0.6;         /* App. B: fac_add */
    p->T_add = 0.002;         /* App. B: T_quality^add */
    p->n_total = 0;           /* no point addition */
}

static int point_cell(const om_mesh* m, double x, double y, int* gi, int* gj) {
    double tx = (x - m->sdf.x0) / m->sdf.dx, ty = (y - m->sdf.y0) / m->sdf.dy;
    double fi = floor(tx), fj = floor(ty);
    int inside = fi >= 0.0 && fi <= (double)(m->ncx - 1) && fj >= 0.0 && fj <= (double)(m->ncy - 1);
    int ii, jj;
    if (!(fi >= 0.0)) ii = 0; else if (fi > (double)(m->ncx - 1)) ii = m->ncx - 1; else ii = (int)fi;
    if (!(fj >= 0.0)) jj = 0; else if (fj > (double)(m->ncy - 1)) jj = m->ncy - 1; else jj = (int)fj;
    *gi = ii; *gj = jj;
    return inside;
}

int om_point_cell(const om_mesh* m, double x, double y, int32_t* gi, int32_t* gj) {
    int a, b;
    int r = point_cell(m, x, y, &a, &b);
    *gi = a; *gj = b;
    return r;
}

static size_t cidx(const om_mesh* m, int gi, int gj) { return (size_t)gj * (size_t)m->ncx + (size_t)gi; }

static double h_at(const om_mesh* m, double x, double y) {
    int gi, gj;
    point_cell(m, x, y, &gi, &gj);
    return m->gh[cidx(m, gi, gj)];
}

/* Sec. 3.2 grid classes; Sec. 3.4/3.5 density; Sec. 3.7 h_i and geps_i. */
static int geometry_setup(om_mesh* m) {
    int ncx = m->sdf.nx - 1, ncy = m->sdf.ny - 1;
    m->ncx = ncx; m->ncy = ncy;
    size_t nc = (size_t)ncx * (size_t)ncy;
    m->gcls = (uint8_t*)malloc(nc);
    m->gh = (double*)malloc(nc * sizeof(double));
    m->ggeps = (double*)malloc(nc * sizeof(double));
    double* rho = (double*)malloc(nc * sizeof(double));
    uint8_t* sel = (uint8_t*)malloc(nc);
    if (!m->gcls || !m->gh || !m->ggeps || !rho || !sel) { free(rho); free(sel); return -1; }
    double dx = m->sdf.dx, dy = m->sdf.dy;
    m->ldiag = sqrt(dx * dx + dy * dy);
    double band = m->P.eta * fmin(dx, dy);
    double sum_rho = 0.0;
    int64_t nsel = 0;
    for (int gj = 0; gj < ncy; gj++)
        for (int gi = 0; gi < ncx; gi++) {
            size_t c = cidx(m, gi, gj);
            const float* r0 = m->sdf.v + (size_t)gj * m->sdf.nx + gi;
            const float* r1 = r0 + m->sdf.nx;
            double sm = 0.25 * ((((double)r0[0] + (double)r0[1]) + (double)r1[0]) + (double)r1[1]);
            uint8_t k = fabs(sm) <= m->ldiag ? CLS_BOUNDARY : (sm < 0.0 ? CLS_INNER : CLS_OUTER);
            m->gcls[c] = k;
            double mx = m->sdf.x0 + ((double)gi + 0.5) * dx;
            double my = m->sdf.y0 + ((double)gj + 0.5) * dy;
            double mu = bilin(&m->siz, mx, my);
            rho[c] = 1.0 / (mu * mu);
            sel[c] = (k == CLS_INNER) || (k == CLS_BOUNDARY && sm <= band);
            if (sel[c]) { sum_rho += rho[c]; nsel++; }
        }
    if (nsel == 0) { free(rho); free(sel); set_err("no inner or selected boundary cells"); return -2; }
    double sum_h = 0.0;
    for (int gj = 0; gj < ncy; gj++)
        for (int gi = 0; gi < ncx; gi++) {
            size_t c = cidx(m, gi, gj);
            double nE = (rho[c] / sum_rho) * (double)m->N;
            m->gh[c] = sqrt((dx * dy) / nE);
            if (sel[c]) sum_h += m->gh[c];
        }
    m->havg = sum_h / (double)nsel;
    for (size_t c = 0; c < nc; c++) m->ggeps[c] = m->P.fac_geps * fmin(m->gh[c], m->havg);
    free(rho);
    free(sel);
    return 0;
}

void om_get_geometry(const om_mesh* m, uint8_t* cls, double* h, double* geps, double* havg) {
    size_t nc = (size_t)m->ncx * (size_t)m->ncy;
    if (cls) memcpy(cls, m->gcls, nc);
    if (h) memcpy(h, m->gh, nc * sizeof(double));
    if (geps) memcpy(geps, m->ggeps, nc * sizeof(double));
    if (havg) *havg = m->havg;
}

/* Sec. 4.3: inner / boundary / outside classification of a point */
static int classify(const om_mesh* m, double x, double y) {
    int gi, gj;
    if (!point_cell(m, x, y, &gi, &gj)) return PT_OUTSIDE;
    size_t c = cidx(m, gi, gj);
    if (m->gcls[c] == CLS_OUTER) return PT_OUTSIDE;
    if (m->gcls[c] == CLS_INNER) return PT_INNER;
    double s = bilin(&m->sdf, x, y), g = m->ggeps[c];
    if (fabs(s) <= g) return PT_BOUNDARY;
    if (s < -g) return PT_INNER;
    return PT_OUTSIDE;
}

om_mesh* om_create(const om_grid* sdf, const om_grid* sizing, const double* xy, int64_t n, const om_params* p) {
    if (n < 0 || (n > 0 && !xy)) { set_err("bad points"); return NULL; }
    om_mesh* m = (om_mesh*)calloc(1, sizeof *m);
    if (!m) return NULL;
    if (p) m->P = *p; else om_default_params(&m->P);
    m->N = n;
    m->Ntot = m->P.n_total > n ? m->P.n_total : n;
    if (!(m->P.fac_add > 0.0)) { set_err("fac_add must be > 0"); om_destroy(m); return NULL; }
    if (grid_copy(&m->sdf, sdf) || grid_copy(&m->siz, sizing)) { set_err("bad grid"); om_destroy(m); return NULL; }
    size_t ns = (size_t)m->siz.nx * (size_t)m->siz.ny;
    for (size_t k = 0; k < ns; k++)
        if (!(m->siz.v[k] > 0.0f)) { set_err("sizing must be positive"); om_destroy(m); return NULL; }
    size_t nn = (size_t)(m->Ntot > 0 ? m->Ntot : 1);
    m->x = (double*)malloc(nn * sizeof(double));
    m->y = (double*)malloc(nn * sizeof(double));
    m->cls = (uint8_t*)malloc(nn);
    m->dprev = (double*)malloc(nn * sizeof(double));
    m->pnew = (double*)calloc(2 * nn, sizeof(double));
    m->force = (double*)calloc(2 * nn, sizeof(double));
    m->fsum = (double*)calloc(nn, sizeof(double));
    m->cen = (double*)calloc(2 * nn, sizeof(double));
    m->area = (double*)calloc(nn, sizeof(double));
    m->qlevel = (int32_t*)calloc(nn, sizeof(int32_t));
    m->ring_off = (int64_t*)calloc(nn + 1, sizeof(int64_t));
    m->tx = (double*)calloc(nn, sizeof(double));
    m->ty = (double*)calloc(nn, sizeof(double));
    m->retri = 1;
    m->threads = 1;
    if (!m->x || !m->y || !m->cls || !m->dprev || !m->pnew || !m->force || !m->fsum || !m->cen || !m->area ||
        !m->qlevel || !m->ring_off || !m->tx || !m->ty) { set_err("out of memory"); om_destroy(m); return NULL; }
    for (int64_t i = 0; i < n; i++) {
        double x = xy[2 * i], y = xy[2 * i + 1];
        if (!isfinite(x) || !isfinite(y) || x < m->sdf.x0 || x > m->sdf.x1 || y < m->sdf.y0 || y > m->sdf.y1) {
            set_err("point not finite or outside the grid box");
            om_destroy(m);
            return NULL;
        }
        m->x[i] = x;
        m->y[i] = y;
    }
    int g = geometry_setup(m);
    if (g) { if (g == -1) set_err("geometry setup failed"); om_destroy(m); return NULL; }
    for (int64_t i = 0; i < n; i++) {
        int c = classify(m, m->x[i], m->y[i]);
        m->cls[i] = c == PT_INNER ? PT_INNER : PT_BOUNDARY; /* reading: outside at init counts as boundary */
        m->dprev[i] = h_at(m, m->x[i], m->y[i]);           /* reading: eps_c = 1 at the first iteration */
    }
    return m;
}

void om_destroy(om_mesh* m) {
    if (!m) return;
    free(m->x); free(m->y); free(m->cls); free(m->dprev);
    free(m->sdf.v); free(m->siz.v);
    free(m->gcls); free(m->gh); free(m->ggeps);
    free(m->ring_off); free(m->ring); free(m->tri); free(m->edge);
    free(m->pnew); free(m->force); free(m->fsum); free(m->cen); free(m->area); free(m->qlevel);
    free(m->tx); free(m->ty);
    free(m);
}

/* ------------------------------------------------------------------------ */
/* Bounded Voronoi cell by half-plane clipping (Sec. 2.1 Fig. 3, Sec. 4.1). */
/* The cell starts as an octagon (enlarged by 1/8 over the span S) cut by    */
/* the (enlarged) domain box; each neighbour, nearest first, cuts it by its  */
/* bisector.  A vertex where two bisectors meet is tested with the exact    */
/* SoS incircle; other vertices with a double power test.  The enlargement  */
/* keeps those inexact decisions away from the region that the triangle     */
/* emission test (on the unenlarged octagon) reads.                         */
/* ------------------------------------------------------------------------ */
static const double RT = 0.70710678118654752440; /* double nearest sqrt(2)/2 */

typedef struct { int64_t j; double d2; } cand_t;

static int cand_cmp(const void* a, const void* b) {
    const cand_t* p = (const cand_t*)a;
    const cand_t* q = (const cand_t*)b;
    if (p->d2 < q->d2) return -1;
    if (p->d2 > q->d2) return 1;
    return p->j < q->j ? -1 : (p->j > q->j ? 1 : 0);
}

static void isect(const hp_t* a, const hp_t* b, double* ux, double* uy, double* det) {
    double D = a->nx * b->ny - a->ny * b->nx;
    *det = D;
    *ux = (a->s * b->ny - b->s * a->ny) / D;
    *uy = (b->s * a->nx - a->s * b->nx) / D;
}

/* upper bound on |vertex|, clipped to the bound RB of the whole polygon */
static double vert_bound(const hp_t* a, const hp_t* b, double RB) {
    double ux, uy, D;
    isect(a, b, &ux, &uy, &D);
    if (D == 0.0) return RB;
    double r = sqrt(ux * ux + uy * uy);
    double err = 1e-9 * (fabs(a->s * b->ny) + fabs(b->s * a->ny) + fabs(b->s * a->nx) + fabs(a->s * b->nx) +
                         r * (fabs(a->nx * b->ny) + fabs(a->ny * b->nx))) / fabs(D);
    if (!(r + err < RB)) return RB;
    return r + err;
}

/* replace the cut run of a convex polygon by the new edge; returns new size,
 * 0 if every vertex was cut, -1 if the cut set was not one run */
static int replace_run(hp_t* E, int ne, const int* cut, const hp_t* l) {
    int ncut = 0, trans = 0, s = -1;
    for (int t = 0; t < ne; t++) {
        ncut += cut[t];
        if (cut[t] && !cut[(t + ne - 1) % ne]) { trans++; s = t; }
    }
    if (ncut == 0) return ne;
    if (ncut == ne) return 0;
    int err = trans != 1;
    int e = s;
    while (cut[e]) e = (e + 1) % ne;
    hp_t tmp[CELL_CAP];
    int k = 0;
    for (int t = e;; t = (t + 1) % ne) {
        tmp[k++] = E[t];
        if (t == s) break;
    }
    tmp[k++] = *l;
    if (k > CELL_CAP) return -2;
    memcpy(E, tmp, sizeof(hp_t) * (size_t)k);
    return err ? -(k + 10) : k;
}

/* floating-point clip: vertex cut iff n.V > s */
static int clip_fp(hp_t* E, int ne, const hp_t* l) {
    int cut[CELL_CAP];
    for (int t = 0; t < ne; t++) {
        double ux, uy, D;
        isect(&E[t], &E[(t + 1) % ne], &ux, &uy, &D);
        cut[t] = (l->nx * ux + l->ny * uy) > l->s;
    }
    return replace_run(E, ne, cut, l);
}

/* simple bucket grid over the domain box for neighbour searches */
typedef struct {
    int nbx, nby;
    double x0, y0, bs;
    int64_t *start, *idx;
} ogrid_t;

static void ogrid_build(const om_mesh* m, ogrid_t* G) {
    double W = m->sdf.x1 - m->sdf.x0, H = m->sdf.y1 - m->sdf.y0;
    double n = m->N > 0 ? (double)m->N : 1.0;
    double bs = sqrt(W * H * 4.0 / n);
    G->nbx = (int)ceil(W / bs); G->nby = (int)ceil(H / bs);
    if (G->nbx < 1) G->nbx = 1;
    if (G->nby < 1) G->nby = 1;
    G->x0 = m->sdf.x0; G->y0 = m->sdf.y0; G->bs = bs;
    size_t nb = (size_t)G->nbx * G->nby;
    G->start = (int64_t*)calloc(nb + 1, sizeof(int64_t));
    G->idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m->N > 0 ? m->N : 1));
    int64_t* key = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m->N > 0 ? m->N : 1));
    for (int64_t i = 0; i < m->N; i++) {
        int bx = (int)floor((m->x[i] - G->x0) / bs), by = (int)floor((m->y[i] - G->y0) / bs);
        if (bx < 0) bx = 0; if (bx >= G->nbx) bx = G->nbx - 1;
        if (by < 0) by = 0; if (by >= G->nby) by = G->nby - 1;
        key[i] = (int64_t)by * G->nbx + bx;
        G->start[key[i] + 1]++;
    }
    for (size_t b = 0; b < nb; b++) G->start[b + 1] += G->start[b];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * nb);
    memcpy(fill, G->start, sizeof(int64_t) * nb);
    for (int64_t i = 0; i < m->N; i++) G->idx[fill[key[i]]++] = i;
    free(fill);
    free(key);
}

static void ogrid_free(ogrid_t* G) { free(G->start); free(G->idx); }

/* Compute the edge list of cell i.  Returns the edge count (0 = empty cell). */
static int cell_compute(const om_mesh* m, const ogrid_t* G, int64_t i, hp_t* E, int64_t* errs) {
    double px = m->x[i], py = m->y[i];
    double pp[2] = {px, py};
    double S = m->P.fac_voro_bound * h_at(m, px, py);
    double W = m->sdf.x1 - m->sdf.x0, H = m->sdf.y1 - m->sdf.y0;
    double SB, RB, mb;
    int ne;
    if (m->P.bounded) {
        SB = S * 1.125;
        RB = SB / cos(M_PI / 8.0) * (1.0 + 1e-9);
        mb = S * 0.125;
        for (int k = 0; k < 8; k++) {
            double c = (k == 0) ? 1.0 : (k == 2 || k == 6) ? 0.0 : (k == 4) ? -1.0 : (k == 1 || k == 7) ? RT : -RT;
            double s = (k == 2) ? 1.0 : (k == 0 || k == 4) ? 0.0 : (k == 6) ? -1.0 : (k == 1 || k == 3) ? RT : -RT;
            E[k].nx = c; E[k].ny = s; E[k].s = SB; E[k].lab = -1 - k;
        }
        ne = 8;
    } else {
        mb = 0.125 * (W > H ? W : H);
        SB = 0.0;
        RB = (sqrt(W * W + H * H) + 4.0 * mb) * (1.0 + 1e-9);
        ne = 0;
    }
    hp_t box[4];
    box[0].nx = -1; box[0].ny = 0; box[0].s = px - (m->sdf.x0 - mb); box[0].lab = -9;
    box[1].nx = 1;  box[1].ny = 0; box[1].s = (m->sdf.x1 + mb) - px; box[1].lab = -10;
    box[2].nx = 0;  box[2].ny = -1; box[2].s = py - (m->sdf.y0 - mb); box[2].lab = -11;
    box[3].nx = 0;  box[3].ny = 1; box[3].s = (m->sdf.y1 + mb) - py; box[3].lab = -12;
    if (m->P.bounded) {
        for (int b = 0; b < 4; b++) {
            int r = clip_fp(E, ne, &box[b]);
            if (r < 0) { (*errs)++; r = r < -2 ? -r - 10 : 0; }
            ne = r;
        }
    } else {
        E[0] = box[2]; E[1] = box[1]; E[2] = box[3]; E[3] = box[0]; /* CCW: bottom right top left */
        ne = 4;
    }
    if (ne == 0) return 0;
    hp_t init[CELL_CAP];
    int ne0 = ne;
    memcpy(init, E, sizeof(hp_t) * (size_t)ne);

    double r = 4.0 * S / m->P.fac_voro_bound; /* start at about four local spacings */
    if (!m->P.bounded) r = 4.0 * sqrt(W * H / (double)(m->N > 0 ? m->N : 1));
    cand_t* C = NULL;
    size_t ccap = 0;
    for (;;) {
        int final_r = 0;
        if (r >= 2.0 * RB) { r = 2.0 * RB * (1.0 + 1e-12); final_r = 1; }
        /* collect candidates within r */
        size_t nc = 0;
        int bx0 = (int)floor((px - r - G->x0) / G->bs), bx1 = (int)floor((px + r - G->x0) / G->bs);
        int by0 = (int)floor((py - r - G->y0) / G->bs), by1 = (int)floor((py + r - G->y0) / G->bs);
        if (bx0 < 0) bx0 = 0; if (by0 < 0) by0 = 0;
        if (bx1 >= G->nbx) bx1 = G->nbx - 1; if (by1 >= G->nby) by1 = G->nby - 1;
        for (int by = by0; by <= by1; by++)
            for (int bx = bx0; bx <= bx1; bx++) {
                size_t b = (size_t)by * G->nbx + bx;
                for (int64_t q = G->start[b]; q < G->start[b + 1]; q++) {
                    int64_t j = G->idx[q];
                    if (j == i) continue;
                    double dx = m->x[j] - px, dy = m->y[j] - py;
                    double d2 = dx * dx + dy * dy;
                    if (d2 < r * r) {
                        if (nc == ccap) { ccap = ccap ? 2 * ccap : 256; C = (cand_t*)realloc(C, ccap * sizeof(cand_t)); }
                        C[nc].j = j; C[nc].d2 = d2; nc++;
                    }
                }
            }
        qsort(C, nc, sizeof(cand_t), cand_cmp);
        ne = ne0;
        memcpy(E, init, sizeof(hp_t) * (size_t)ne);
        double Rmax = 0.0;
        for (int t = 0; t < ne; t++) {
            double b = vert_bound(&E[t], &E[(t + 1) % ne], RB);
            if (b > Rmax) Rmax = b;
        }
        int closed = 0, empty = 0;
        for (size_t q = 0; q < nc; q++) {
            int64_t l = C[q].j;
            double dx = m->x[l] - px, dy = m->y[l] - py;
            if (dx == 0.0 && dy == 0.0) {
                if (l > i) { empty = 1; break; } /* SoS: the higher id owns a duplicate site */
                continue;
            }
            if (sqrt(C[q].d2) >= 2.0 * Rmax) { closed = 1; break; }
            /* a site with an exact duplicate of larger id has an empty cell under
             * SoS; its bisector is dominated by the duplicate's, so skip it */
            int dominated = 0;
            for (size_t q2 = 0; q2 < nc && C[q2].d2 <= C[q].d2; q2++)
                if (C[q2].d2 == C[q].d2 && C[q2].j > l && m->x[C[q2].j] == m->x[l] && m->y[C[q2].j] == m->y[l])
                    dominated = 1;
            if (dominated) continue;
            hp_t hl;
            hl.nx = dx; hl.ny = dy; hl.s = 0.5 * (dx * dx + dy * dy); hl.lab = (int32_t)l;
            int cut[CELL_CAP];
            double pl[2] = {m->x[l], m->y[l]};
            for (int t = 0; t < ne; t++) {
                const hp_t* a = &E[t];
                const hp_t* b = &E[(t + 1) % ne];
                if (a->lab >= 0 && b->lab >= 0) {
                    double pa[2] = {m->x[a->lab], m->y[a->lab]}, pb[2] = {m->x[b->lab], m->y[b->lab]};
                    int o = om_orient2d(pp, pa, pb);
                    int s = om_incircle_sos(pp, i, pa, a->lab, pb, b->lab, pl, l);
                    if (o == 0) (*errs)++;
                    cut[t] = (s * o) > 0;
                } else {
                    double ux, uy, D;
                    isect(a, b, &ux, &uy, &D);
                    cut[t] = (hl.nx * ux + hl.ny * uy) > hl.s;
                }
            }
            int rr = replace_run(E, ne, cut, &hl);
            if (rr == -2) { (*errs)++; empty = 1; break; }
            if (rr < 0) { (*errs)++; rr = -rr - 10; }
            if (rr == 0) { empty = 1; break; }
            ne = rr;
            Rmax = 0.0;
            for (int t = 0; t < ne; t++) {
                double b = vert_bound(&E[t], &E[(t + 1) % ne], RB);
                if (b > Rmax) Rmax = b;
            }
        }
        if (empty) { free(C); return 0; }
        if (closed || final_r || 2.0 * Rmax <= r) break;
        r *= 2.0;
    }
    free(C);
    return ne;
}

/* ------------------------------------------------------------------------ */
/* Triangle emission (Sec. 4.1) with the fixed FP64 formulas                */
/* ------------------------------------------------------------------------ */
/* circumcentre of (a,b,c) computed from a; canonical a = smallest id, a,b,c CCW */
static void circumcenter_fixed(double ax, double ay, double bx_, double by_, double cx_, double cy_,
                               double* ox, double* oy, double* R) {
    double bx = bx_ - ax, by = by_ - ay, cx = cx_ - ax, cy = cy_ - ay;
    double B = bx * bx + by * by;
    double C = cx * cx + cy * cy;
    double D = 2.0 * (bx * cy - by * cx);
    double ux = (cy * B - by * C) / D;
    double uy = (bx * C - cx * B) / D;
    *ox = ax + ux;
    *oy = ay + uy;
    *R = sqrt(ux * ux + uy * uy);
}

/* c in Reg_i = Oct_i (span S_i) intersected with the domain box */
static int reg_contains(const om_mesh* m, int64_t i, double cx, double cy) {
    if (!(cx >= m->sdf.x0 && cx <= m->sdf.x1 && cy >= m->sdf.y0 && cy <= m->sdf.y1)) return 0;
    if (!m->P.bounded) return 1;
    double S = m->P.fac_voro_bound * h_at(m, m->x[i], m->y[i]);
    double dx = cx - m->x[i], dy = cy - m->y[i];
    return fabs(dx) <= S && fabs(dy) <= S && fabs(RT * (dx + dy)) <= S && fabs(RT * (dy - dx)) <= S;
}

/* Tests 1-3 of Sec. 4.1 on the bilinear SDF grid */
static int triangle_valid(const om_mesh* m, int64_t a, int64_t b, int64_t c) {
    double ax = m->x[a], ay = m->y[a], bx = m->x[b], by = m->y[b], cx = m->x[c], cy = m->y[c];
    int gi, gj;
    double gx = ((ax + bx) + cx) / 3.0, gy = ((ay + by) + cy) / 3.0;
    if (!point_cell(m, gx, gy, &gi, &gj)) return 0;
    size_t cc = cidx(m, gi, gj);
    if (m->gcls[cc] == CLS_INNER) return 1;
    if (m->gcls[cc] == CLS_OUTER) return 0;
    if (bilin(&m->sdf, gx, gy) > m->ggeps[cc]) return 0;
    int count = 0;
    double mids[3][2] = {{(ax + bx) * 0.5, (ay + by) * 0.5}, {(bx + cx) * 0.5, (by + cy) * 0.5},
                         {(cx + ax) * 0.5, (cy + ay) * 0.5}};
    for (int k = 0; k < 3; k++) {
        if (!point_cell(m, mids[k][0], mids[k][1], &gi, &gj)) continue;
        size_t q = cidx(m, gi, gj);
        if (m->gcls[q] == CLS_INNER) count++;
        else if (m->gcls[q] == CLS_BOUNDARY && bilin(&m->sdf, mids[k][0], mids[k][1]) <= m->ggeps[q]) count++;
    }
    if (count >= 2) return 1;
    double ox, oy, R;
    circumcenter_fixed(ax, ay, bx, by, cx, cy, &ox, &oy, &R);
    return fabs(bilin(&m->sdf, ox, oy)) / R <= m->P.T_circ;
}

static int tri_cmp(const void* a, const void* b) {
    const int32_t* p = (const int32_t*)a;
    const int32_t* q = (const int32_t*)b;
    for (int k = 0; k < 3; k++)
        if (p[k] != q[k]) return p[k] < q[k] ? -1 : 1;
    return 0;
}

static int edge_cmp(const void* a, const void* b) {
    const int32_t* p = (const int32_t*)a;
    const int32_t* q = (const int32_t*)b;
    for (int k = 0; k < 2; k++)
        if (p[k] != q[k]) return p[k] < q[k] ? -1 : 1;
    return 0;
}

/* Procedure I over all cells on m->threads threads: thread t clips the
 * contiguous cells [N t / T, N (t+1) / T) into its own buffer, and the
 * buffers are concatenated in cell order, so the rings are those of one
 * thread */
static void rebuild_all_cells_mt(om_mesh* m, const ogrid_t* G) {
    int T = m->threads;
    int32_t** buf = (int32_t**)calloc((size_t)T, sizeof(int32_t*));
    int64_t* len = (int64_t*)calloc((size_t)T, sizeof(int64_t));
    int64_t errs = 0;
#pragma omp parallel num_threads(T) reduction(+ : errs)
    {
        int t = omp_get_thread_num();
        int64_t lo = m->N * t / T, hi = m->N * (t + 1) / T, cap = 8 * (hi - lo) + 64, n = 0;
        int32_t* b = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
        hp_t E[CELL_CAP];
        for (int64_t i = lo; i < hi; i++) {
            int ne = cell_compute(m, G, i, E, &errs);
            if (n + ne > cap) {
                cap = 2 * (n + ne);
                b = (int32_t*)realloc(b, sizeof(int32_t) * (size_t)cap);
            }
            for (int k = 0; k < ne; k++) b[n + k] = E[k].lab;
            n += ne;
            m->ring_off[i + 1] = ne; /* counts; offsets below */
        }
        buf[t] = b;
        len[t] = n;
    }
    int64_t total = 0;
    for (int t = 0; t < T; t++) total += len[t];
    free(m->ring);
    m->ring_cap = total > 0 ? total : 1;
    m->ring = (int32_t*)malloc(sizeof(int32_t) * (size_t)m->ring_cap);
    m->ring_off[0] = 0;
    for (int64_t i = 0; i < m->N; i++) m->ring_off[i + 1] += m->ring_off[i];
    for (int t = 0; t < T; t++) {
        int64_t lo = m->N * t / T;
        memcpy(m->ring + m->ring_off[lo], buf[t], sizeof(int32_t) * (size_t)len[t]);
        free(buf[t]);
    }
    free(buf);
    free(len);
    m->clip_errors = errs;
}

/* Procedure I */
static int rebuild_cells(om_mesh* m, const int64_t* cells, int64_t ncells, int keep) {
    ogrid_t G;
    ogrid_build(m, &G);
    if (keep && !cells && m->threads > 1) {
        rebuild_all_cells_mt(m, &G);
        ogrid_free(&G);
        return 0;
    }
    hp_t E[CELL_CAP];
    int64_t errs = 0;
    int64_t total = 0;
    int64_t ncalc = cells ? ncells : m->N;
    if (keep) {
        free(m->ring);
        m->ring_cap = 8 * (m->N > 0 ? m->N : 1);
        m->ring = (int32_t*)malloc(sizeof(int32_t) * (size_t)m->ring_cap);
        m->ring_off[0] = 0;
    }
    for (int64_t q = 0; q < ncalc; q++) {
        int64_t i = cells ? cells[q] : q;
        int ne = cell_compute(m, &G, i, E, &errs);
        if (keep) {
            if (total + ne > m->ring_cap) {
                m->ring_cap = 2 * (total + ne);
                m->ring = (int32_t*)realloc(m->ring, sizeof(int32_t) * (size_t)m->ring_cap);
            }
            for (int t = 0; t < ne; t++) m->ring[total + t] = E[t].lab;
            total += ne;
            m->ring_off[i + 1] = total;
        }
    }
    ogrid_free(&G);
    m->clip_errors = errs;
    return 0;
}

/* the valid triangles owned (smallest index) by cells [lo, hi), appended
 * to *tri (capacity *cap, count *nt) */
static void emit_range(const om_mesh* m, int64_t lo, int64_t hi, int32_t** tri, int64_t* cap, int64_t* nt) {
    for (int64_t i = lo; i < hi; i++) {
        int64_t o = m->ring_off[i], ne = m->ring_off[i + 1] - o;
        for (int64_t t = 0; t < ne; t++) {
            int32_t j = m->ring[o + t], k = m->ring[o + (t + 1) % ne];
            if (j < 0 || k < 0 || !(i < j && i < k)) continue;
            double ox, oy, R;
            circumcenter_fixed(m->x[i], m->y[i], m->x[j], m->y[j], m->x[k], m->y[k], &ox, &oy, &R);
            if (!(reg_contains(m, i, ox, oy) && reg_contains(m, j, ox, oy) && reg_contains(m, k, ox, oy))) continue;
            if (m->P.validity && !triangle_valid(m, i, j, k)) continue;
            if (*nt == *cap) { *cap *= 2; *tri = (int32_t*)realloc(*tri, sizeof(int32_t) * 3 * (size_t)*cap); }
            (*tri)[3 * *nt] = (int32_t)i; (*tri)[3 * *nt + 1] = j; (*tri)[3 * *nt + 2] = k;
            (*nt)++;
        }
    }
}

static int emit_triangles(om_mesh* m) {
    int64_t cap = 2 * m->N + 16, nt = 0;
    free(m->tri);
    m->tri = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)cap);
    if (m->threads > 1) {
        /* per-thread lists, concatenated; the sort below fixes the order */
        int T = m->threads;
        int32_t** buf = (int32_t**)calloc((size_t)T, sizeof(int32_t*));
        int64_t* cnt = (int64_t*)calloc((size_t)T, sizeof(int64_t));
#pragma omp parallel num_threads(T)
        {
            int t = omp_get_thread_num();
            int64_t lo = m->N * t / T, hi = m->N * (t + 1) / T, c = 2 * (hi - lo) + 16, n = 0;
            int32_t* b = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)c);
            emit_range(m, lo, hi, &b, &c, &n);
            buf[t] = b;
            cnt[t] = n;
        }
        for (int t = 0; t < T; t++) {
            if (nt + cnt[t] > cap) {
                cap = 2 * (nt + cnt[t]);
                m->tri = (int32_t*)realloc(m->tri, sizeof(int32_t) * 3 * (size_t)cap);
            }
            memcpy(m->tri + 3 * nt, buf[t], sizeof(int32_t) * 3 * (size_t)cnt[t]);
            nt += cnt[t];
            free(buf[t]);
        }
        free(buf);
        free(cnt);
    } else {
        emit_range(m, 0, m->N, &m->tri, &cap, &nt);
    }
    qsort(m->tri, (size_t)nt, 3 * sizeof(int32_t), tri_cmp);
    m->ntri = nt;
    /* unique edges of valid triangles */
    free(m->edge);
    m->edge = (int32_t*)malloc(sizeof(int32_t) * 6 * (size_t)(nt > 0 ? nt : 1));
    int64_t ne = 0;
    for (int64_t t = 0; t < nt; t++)
        for (int k = 0; k < 3; k++) {
            int32_t a = m->tri[3 * t + k], b = m->tri[3 * t + (k + 1) % 3];
            m->edge[2 * ne] = a < b ? a : b;
            m->edge[2 * ne + 1] = a < b ? b : a;
            ne++;
        }
    qsort(m->edge, (size_t)ne, 2 * sizeof(int32_t), edge_cmp);
    int64_t u = 0;
    for (int64_t e = 0; e < ne; e++)
        if (u == 0 || m->edge[2 * e] != m->edge[2 * (u - 1)] || m->edge[2 * e + 1] != m->edge[2 * (u - 1) + 1]) {
            m->edge[2 * u] = m->edge[2 * e];
            m->edge[2 * u + 1] = m->edge[2 * e + 1];
            u++;
        }
    m->nedge = u;
    return 0;
}

/* sum of v[0..n) by pairwise (cascade) summation in index order: the
 * rounding of the result grows like log2(n) ulps rather than n */
static double pairwise_sum(const double* v, int64_t n) {
    if (n <= 8) {
        double s = 0.0;
        for (int64_t k = 0; k < n; k++) s += v[k];
        return s;
    }
    int64_t h = n / 2;
    return pairwise_sum(v, h) + pairwise_sum(v + h, n - h);
}

/* Eq. 3 over the valid edges at the current positions: fac_mu =
 * sqrt(sum l^2 / sum mu(m)^2), both sums pairwise in edge order */
static double eq3_fac_mu(const om_mesh* m) {
    if (m->nedge <= 0) return 1.0;
    double* t = (double*)malloc(sizeof(double) * 2 * (size_t)m->nedge);
    double *tl = t, *tm = t + m->nedge;
    for (int64_t e = 0; e < m->nedge; e++) {
        int32_t i = m->edge[2 * e], j = m->edge[2 * e + 1];
        double dx = m->x[j] - m->x[i], dy = m->y[j] - m->y[i];
        double mu = bilin(&m->siz, (m->x[i] + m->x[j]) * 0.5, (m->y[i] + m->y[j]) * 0.5);
        tl[e] = dx * dx + dy * dy;
        tm[e] = mu * mu;
    }
    double f = sqrt(pairwise_sum(tl, m->nedge) / pairwise_sum(tm, m->nedge));
    free(t);
    return f;
}

/* Sec. 3.6 Eq. 11-12 and Sec. 2.2 Eq. 3 */
static void quality(om_mesh* m) {
    double sa = 0, sb = 0, amax = 0, bmax = 0, minang = 180.0;
    for (int64_t t = 0; t < m->ntri; t++) {
        int32_t a = m->tri[3 * t], b = m->tri[3 * t + 1], c = m->tri[3 * t + 2];
        double la = hypot(m->x[b] - m->x[c], m->y[b] - m->y[c]);
        double lb = hypot(m->x[c] - m->x[a], m->y[c] - m->y[a]);
        double lc = hypot(m->x[a] - m->x[b], m->y[a] - m->y[b]);
        double o = (m->x[b] - m->x[a]) * (m->y[c] - m->y[a]) - (m->y[b] - m->y[a]) * (m->x[c] - m->x[a]);
        double A = 0.5 * fabs(o);
        double alpha = (la * lb * lc * (la + lb + lc)) / (16.0 * A * A);
        double lmax = fmax(la, fmax(lb, lc)), lmin = fmin(la, fmin(lb, lc));
        double beta = lmax / lmin;
        /* smallest angle is opposite the shortest side */
        double p, q;
        if (lmin == la) { p = lb; q = lc; } else if (lmin == lb) { p = la; q = lc; } else { p = la; q = lb; }
        double cs = (p * p + q * q - lmin * lmin) / (2.0 * p * q);
        if (cs > 1.0) cs = 1.0; if (cs < -1.0) cs = -1.0;
        double ang = acos(cs) * (180.0 / M_PI);
        sa += sqrt(alpha);
        sb += sqrt(beta);
        if (alpha > amax) amax = alpha;
        if (beta > bmax) bmax = beta;
        if (ang < minang) minang = ang;
    }
    double n = (double)m->ntri;
    m->st.n_tri = m->ntri;
    m->st.n_edges = m->nedge;
    m->st.half_mean_alpha = n > 0 ? (sa / n) * (sa / n) : 0.0;
    m->st.half_mean_beta = n > 0 ? (sb / n) * (sb / n) : 0.0;
    m->st.max_alpha = amax;
    m->st.max_beta = bmax;
    m->st.min_angle_deg = n > 0 ? minang : 0.0;
    /* fac_mu over the valid edges (Eq. 3) */
    m->st.fac_mu = eq3_fac_mu(m);
    double dev = 0;
    for (int64_t e = 0; e < m->nedge; e++) {
        int32_t i = m->edge[2 * e], j = m->edge[2 * e + 1];
        double dx = m->x[j] - m->x[i], dy = m->y[j] - m->y[i];
        double mu = bilin(&m->siz, (m->x[i] + m->x[j]) * 0.5, (m->y[i] + m->y[j]) * 0.5);
        dev += fabs(sqrt(dx * dx + dy * dy) / (m->st.fac_mu * mu) - 1.0);
    }
    m->st.mean_size_dev = m->nedge > 0 ? dev / (double)m->nedge : 0.0;
}

int om_rebuild(om_mesh* m) {
    rebuild_cells(m, NULL, 0, 1);
    emit_triangles(m);
    quality(m);
    m->st.clip_errors = m->clip_errors;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* DistMesh move (Sec. 2.2, Eqs. 2-5)                                        */
/* ------------------------------------------------------------------------ */
static void distmesh_move(om_mesh* m) {
    memset(m->force, 0, sizeof(double) * 2 * (size_t)m->N);
    memset(m->fsum, 0, sizeof(double) * (size_t)m->N);
    double fac_mu = m->st.fac_mu;
    for (int64_t e = 0; e < m->nedge; e++) {
        int32_t i = m->edge[2 * e], j = m->edge[2 * e + 1];
        double dx = m->x[i] - m->x[j], dy = m->y[i] - m->y[j];
        double l = sqrt(dx * dx + dy * dy);
        double mu = bilin(&m->siz, (m->x[i] + m->x[j]) * 0.5, (m->y[i] + m->y[j]) * 0.5);
        double l0 = m->P.fac_F * fac_mu * mu;
        if (!(l < l0)) continue;
        double f = m->P.k_spring * (l0 - l);
        m->force[2 * i] += f * dx / l;
        m->force[2 * i + 1] += f * dy / l;
        m->force[2 * j] -= f * dx / l;
        m->force[2 * j + 1] -= f * dy / l;
        m->fsum[i] += f;
        m->fsum[j] += f;
    }
    for (int64_t i = 0; i < m->N; i++) {
        m->pnew[2 * i] = m->x[i] + m->P.dt * m->force[2 * i];
        m->pnew[2 * i + 1] = m->y[i] + m->P.dt * m->force[2 * i + 1];
    }
}

/* ------------------------------------------------------------------------ */
/* CVD centroid (Sec. 2.3 Eq. 6, Sec. 4.2)                                   */
/* ------------------------------------------------------------------------ */
/* one-point rule on each leaf of a longest-edge bisection tree of depth d */
static void quad_tri(const grid_t* siz, double gx, double gy, const double* q0, const double* q1, const double* q2,
                     int depth, double* W, double* WX, double* WY) {
    if (depth == 0) {
        double A = 0.5 * ((q1[0] - q0[0]) * (q2[1] - q0[1]) - (q1[1] - q0[1]) * (q2[0] - q0[0]));
        double cx = (q0[0] + q1[0] + q2[0]) / 3.0, cy = (q0[1] + q1[1] + q2[1]) / 3.0;
        double mu = bilin(siz, gx + cx, gy + cy);
        double w = A / (mu * mu);
        *W += w;
        *WX += w * cx;
        *WY += w * cy;
        return;
    }
    double L01 = (q1[0] - q0[0]) * (q1[0] - q0[0]) + (q1[1] - q0[1]) * (q1[1] - q0[1]);
    double L12 = (q2[0] - q1[0]) * (q2[0] - q1[0]) + (q2[1] - q1[1]) * (q2[1] - q1[1]);
    double L20 = (q0[0] - q2[0]) * (q0[0] - q2[0]) + (q0[1] - q2[1]) * (q0[1] - q2[1]);
    const double *a = q0, *b = q1, *c = q2;
    double Lm = L01;
    if (L12 > Lm) { a = q1; b = q2; c = q0; Lm = L12; }
    if (L20 > Lm) { a = q2; b = q0; c = q1; }
    double mid[2] = {(a[0] + b[0]) * 0.5, (a[1] + b[1]) * 0.5};
    quad_tri(siz, gx, gy, a, mid, c, depth - 1, W, WX, WY);
    quad_tri(siz, gx, gy, mid, b, c, depth - 1, W, WX, WY);
}

/* centroid of polygon poly (vertices relative to gen, CCW) by adaptive
 * quadrature; returns 0 when the polygon has no weight */
static int centroid_adaptive(const grid_t* siz, const double* gen, const double* poly, int nv, double eps_c,
                             int max_level, double* c, int32_t* level, double* area_out) {
    double A = 0;
    for (int t = 0; t < nv; t++) {
        const double* v0 = poly + 2 * t;
        const double* v1 = poly + 2 * ((t + 1) % nv);
        A += 0.5 * (v0[0] * v1[1] - v0[1] * v1[0]);
    }
    if (area_out) *area_out = A;
    if (!(A > 0)) { c[0] = gen[0]; c[1] = gen[1]; *level = 0; return 0; }
    double E = sqrt(A) * eps_c;
    double px = 0.0, py = 0.0; /* level 0: the generator itself */
    static const double origin[2] = {0.0, 0.0};
    for (int k = 1; k <= max_level; k++) {
        double W = 0, WX = 0, WY = 0;
        for (int t = 0; t < nv; t++)
            quad_tri(siz, gen[0], gen[1], origin, poly + 2 * t, poly + 2 * ((t + 1) % nv), k - 1, &W, &WX, &WY);
        if (!(W > 0)) { c[0] = gen[0]; c[1] = gen[1]; *level = 0; return 0; }
        double cx = WX / W, cy = WY / W;
        double dx = cx - px, dy = cy - py;
        if (sqrt(dx * dx + dy * dy) < E || k == max_level) {
            c[0] = gen[0] + cx;
            c[1] = gen[1] + cy;
            *level = k;
            return k == max_level && !(sqrt(dx * dx + dy * dy) < E) ? 2 : 1;
        }
        px = cx;
        py = cy;
    }
    return 1;
}

/* V_i = cell of i clipped to Reg_i, vertices relative to p_i */
static int cell_polygon_labels(const om_mesh* m, int64_t i, const int32_t* ring, int64_t ne, double* out, int cap);

static int cell_polygon(const om_mesh* m, int64_t i, double* out, int cap) {
    int64_t o = m->ring_off[i], ne = m->ring_off[i + 1] - o;
    return cell_polygon_labels(m, i, m->ring + o, ne, out, cap);
}

static int cell_polygon_labels(const om_mesh* m, int64_t i, const int32_t* ring, int64_t ne, double* out, int cap) {
    if (ne == 0) return 0;
    hp_t E[CELL_CAP];
    double px = m->x[i], py = m->y[i];
    double S = m->P.fac_voro_bound * h_at(m, px, py);
    double W = m->sdf.x1 - m->sdf.x0, H = m->sdf.y1 - m->sdf.y0;
    double mb = m->P.bounded ? S * 0.125 : 0.125 * (W > H ? W : H);
    for (int64_t t = 0; t < ne; t++) {
        int32_t lab = ring[t];
        hp_t* e = &E[t];
        e->lab = lab;
        if (lab >= 0) {
            e->nx = m->x[lab] - px; e->ny = m->y[lab] - py;
            e->s = 0.5 * (e->nx * e->nx + e->ny * e->ny);
        } else if (lab >= -8) {
            int k = -1 - lab;
            e->nx = (k == 0) ? 1.0 : (k == 2 || k == 6) ? 0.0 : (k == 4) ? -1.0 : (k == 1 || k == 7) ? RT : -RT;
            e->ny = (k == 2) ? 1.0 : (k == 0 || k == 4) ? 0.0 : (k == 6) ? -1.0 : (k == 1 || k == 3) ? RT : -RT;
            e->s = S * 1.125;
        } else {
            int b = -9 - lab;
            e->nx = b == 0 ? -1 : b == 1 ? 1 : 0;
            e->ny = b == 2 ? -1 : b == 3 ? 1 : 0;
            e->s = b == 0 ? px - (m->sdf.x0 - mb) : b == 1 ? (m->sdf.x1 + mb) - px
                 : b == 2 ? py - (m->sdf.y0 - mb) : (m->sdf.y1 + mb) - py;
        }
    }
    int n = (int)ne;
    if (m->P.bounded)
        for (int k = 0; k < 8 && n > 0; k++) {
            hp_t l;
            l.nx = (k == 0) ? 1.0 : (k == 2 || k == 6) ? 0.0 : (k == 4) ? -1.0 : (k == 1 || k == 7) ? RT : -RT;
            l.ny = (k == 2) ? 1.0 : (k == 0 || k == 4) ? 0.0 : (k == 6) ? -1.0 : (k == 1 || k == 3) ? RT : -RT;
            l.s = S; l.lab = -101 - k;
            int r = clip_fp(E, n, &l);
            n = r < 0 ? (r < -2 ? -r - 10 : 0) : r;
        }
    hp_t bl[4];
    bl[0].nx = -1; bl[0].ny = 0; bl[0].s = px - m->sdf.x0; bl[0].lab = -109;
    bl[1].nx = 1; bl[1].ny = 0; bl[1].s = m->sdf.x1 - px; bl[1].lab = -110;
    bl[2].nx = 0; bl[2].ny = -1; bl[2].s = py - m->sdf.y0; bl[2].lab = -111;
    bl[3].nx = 0; bl[3].ny = 1; bl[3].s = m->sdf.y1 - py; bl[3].lab = -112;
    for (int b = 0; b < 4 && n > 0; b++) {
        int r = clip_fp(E, n, &bl[b]);
        n = r < 0 ? (r < -2 ? -r - 10 : 0) : r;
    }
    if (n > cap) n = cap;
    for (int t = 0; t < n; t++) {
        double D;
        isect(&E[t], &E[(t + 1) % n], &out[2 * t], &out[2 * t + 1], &D);
    }
    return n;
}

int om_get_cell_polygon(const om_mesh* m, int64_t i, double* xy, int cap) {
    double buf[2 * CELL_CAP];
    int n = cell_polygon(m, i, buf, CELL_CAP);
    if (n > cap) n = cap;
    for (int t = 0; t < n; t++) { xy[2 * t] = buf[2 * t] + m->x[i]; xy[2 * t + 1] = buf[2 * t + 1] + m->y[i]; }
    return n;
}

int om_get_ring(const om_mesh* m, int64_t i, int32_t* labels, int cap) {
    int64_t o = m->ring_off[i], ne = m->ring_off[i + 1] - o;
    for (int64_t t = 0; t < ne && t < cap; t++) labels[t] = m->ring[o + t];
    return (int)ne;
}

static void cvd_move(om_mesh* m) {
    int64_t qcap = 0;
#pragma omp parallel for num_threads(m->threads > 1 ? m->threads : 1) schedule(dynamic, 1024) reduction(+ : qcap)
    for (int64_t i = 0; i < m->N; i++) {
        double poly[2 * CELL_CAP];
        int n = cell_polygon(m, i, poly, CELL_CAP);
        double gen[2] = {m->x[i], m->y[i]};
        double h = h_at(m, m->x[i], m->y[i]);
        double eps_c = fmax(m->dprev[i] / h, m->P.fac_end);
        int32_t lv = 0;
        double A = 0;
        int r = n >= 3 ? centroid_adaptive(&m->siz, gen, poly, n, eps_c, m->P.quad_max_level, &m->cen[2 * i], &lv, &A)
                       : (m->cen[2 * i] = gen[0], m->cen[2 * i + 1] = gen[1], 0);
        if (r == 2) qcap++;
        m->qlevel[i] = lv;
        m->area[i] = A;
        m->pnew[2 * i] = m->cen[2 * i];
        m->pnew[2 * i + 1] = m->cen[2 * i + 1];
    }
    m->st.quad_cap += qcap;
}

int om_polygon_centroid(const om_grid* sizing, const double* gen, const double* poly, int nv, double eps_c,
                        int max_level, double* c, int32_t* level) {
    grid_t g;
    g.nx = sizing->nx; g.ny = sizing->ny; g.x0 = sizing->x0; g.y0 = sizing->y0; g.x1 = sizing->x1; g.y1 = sizing->y1;
    g.dx = (g.x1 - g.x0) / (double)(g.nx - 1);
    g.dy = (g.y1 - g.y0) / (double)(g.ny - 1);
    g.v = (float*)sizing->v;
    double* rel = (double*)malloc(sizeof(double) * 2 * (size_t)(nv > 0 ? nv : 1));
    for (int t = 0; t < nv; t++) { rel[2 * t] = poly[2 * t] - gen[0]; rel[2 * t + 1] = poly[2 * t + 1] - gen[1]; }
    int r = centroid_adaptive(&g, gen, rel, nv, eps_c, max_level, c, level, NULL);
    free(rel);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Point treatment (Sec. 4.3)                                                */
/* ------------------------------------------------------------------------ */
static double geps_at(const om_mesh* m, double x, double y) {
    int gi, gj;
    point_cell(m, x, y, &gi, &gj);
    return m->ggeps[cidx(m, gi, gj)];
}

/* sphere tracing from an inner p_old toward an outside p_new (Fig. 21a) */
static int sphere_trace(om_mesh* m, const double* a, const double* b, double* out) {
    double Lx = b[0] - a[0], Ly = b[1] - a[1];
    double L = sqrt(Lx * Lx + Ly * Ly);
    double ux = Lx / L, uy = Ly / L;
    double x[2] = {a[0], a[1]}, lo[2] = {a[0], a[1]}, hi[2] = {b[0], b[1]};
    double t = 0.0;
    int it = 0, bisect = 0;
    for (; it < m->P.trace_max; it++) {
        double s = bilin(&m->sdf, x[0], x[1]), g = geps_at(m, x[0], x[1]);
        if (fabs(s) <= g) { out[0] = x[0]; out[1] = x[1]; return 0; }
        if (s > g) { hi[0] = x[0]; hi[1] = x[1]; bisect = 1; break; }
        lo[0] = x[0]; lo[1] = x[1];
        t += fabs(s);
        if (t >= L) { bisect = 1; break; } /* passed p_new, which is outside */
        x[0] = a[0] + t * ux;
        x[1] = a[1] + t * uy;
    }
    if (bisect)
        for (it++; it < m->P.trace_max; it++) {
            double mid[2] = {(lo[0] + hi[0]) * 0.5, (lo[1] + hi[1]) * 0.5};
            double s = bilin(&m->sdf, mid[0], mid[1]), g = geps_at(m, mid[0], mid[1]);
            if (fabs(s) <= g) { out[0] = mid[0]; out[1] = mid[1]; return 0; }
            if (s < 0) { lo[0] = mid[0]; lo[1] = mid[1]; } else { hi[0] = mid[0]; hi[1] = mid[1]; }
        }
    out[0] = lo[0];
    out[1] = lo[1];
    return 1; /* cap hit: last inside point */
}

/* damped Newton projection (Eqs. 8-10); gradient taken at the iterate */
static void newton_project(om_mesh* m, const double* pn, double* out) {
    double x = pn[0], y = pn[1];
    for (int k = 0; k < m->P.newton_max; k++) {
        double f, fx, fy, fxy;
        bilin_d(&m->sdf, x, y, &f, &fx, &fy, &fxy);
        double L1 = f;
        double L2 = (x - pn[0]) * fy - (y - pn[1]) * fx;
        double J00 = fx, J01 = fy;
        double J10 = fy + (x - pn[0]) * fxy, J11 = -fx - (y - pn[1]) * fxy;
        double det = J00 * J11 - J01 * J10;
        if (det == 0.0 || !isfinite(det)) break;
        double dx = (J11 * L1 - J01 * L2) / det;
        double dy = (-J10 * L1 + J00 * L2) / det;
        x -= m->P.damping * dx;
        y -= m->P.damping * dy;
        if (fabs(bilin(&m->sdf, x, y)) <= geps_at(m, x, y)) break;
    }
    out[0] = x;
    out[1] = y;
}

static int treat_point(om_mesh* m, const double* po, int ocls, const double* pn_in, double* pf, int32_t* ncls,
                       int64_t* nfail, int64_t* tcap) {
    double h = h_at(m, po[0], po[1]);
    double dx = pn_in[0] - po[0], dy = pn_in[1] - po[1];
    double d = sqrt(dx * dx + dy * dy);
    double T = m->P.fac_pt * h;
    double pn[2] = {pn_in[0], pn_in[1]};
    if (d > T) { pn[0] = po[0] + dx * (T / d); pn[1] = po[1] + dy * (T / d); }
    int c = classify(m, pn[0], pn[1]);
    if (c != PT_OUTSIDE) { pf[0] = pn[0]; pf[1] = pn[1]; *ncls = c; return 0; }
    double ps[2];
    if (ocls == PT_INNER) {
        if (sphere_trace(m, po, pn, ps)) (*tcap)++;
        int cc = classify(m, ps[0], ps[1]);
        if (cc == PT_OUTSIDE) { pf[0] = po[0]; pf[1] = po[1]; *ncls = ocls; return 1; }
        pf[0] = ps[0]; pf[1] = ps[1]; *ncls = cc;
        return 0;
    }
    newton_project(m, pn, ps);
    if (classify(m, ps[0], ps[1]) == PT_BOUNDARY) { pf[0] = ps[0]; pf[1] = ps[1]; *ncls = PT_BOUNDARY; return 0; }
    (*nfail)++;
    pf[0] = po[0]; pf[1] = po[1]; *ncls = ocls;
    return 1;
}

int om_project_point(om_mesh* m, const double* p_old, int old_class, const double* p_new, double* p_final,
                     int32_t* new_class) {
    int64_t a = 0, b = 0;
    return treat_point(m, p_old, old_class, p_new, p_final, new_class, &a, &b);
}

/* ------------------------------------------------------------------------ */
/* one meshing iteration                                                    */
/* ------------------------------------------------------------------------ */
/* Eq. 3 scaling factor over the stored valid edges at the current positions
 * (a DistMesh step that keeps the last triangulation, Algorithm 1) */
static void fac_mu_current(om_mesh* m) { m->st.fac_mu = eq3_fac_mu(m); }

/* ------------------------------------------------------------------------ */
/* point addition (Sec. 3.6) and the rescaled quantities (Sec. 3.7)         */
/* ------------------------------------------------------------------------ */
typedef struct {
    double ratio;     /* R_circ / h_i */
    int32_t v[3];     /* vertex indices, ascending */
    double gx, gy;    /* centroid */
} addc_t;

/* larger ratio first; equal ratios by the smaller vertex triple */
static int addc_rank_cmp(const void* a, const void* b) {
    const addc_t* p = (const addc_t*)a;
    const addc_t* q = (const addc_t*)b;
    if (p->ratio != q->ratio) return p->ratio > q->ratio ? -1 : 1;
    for (int k = 0; k < 3; k++)
        if (p->v[k] != q->v[k]) return p->v[k] < q->v[k] ? -1 : 1;
    return 0;
}

static int addc_triple_cmp(const void* a, const void* b) {
    const addc_t* p = (const addc_t*)a;
    const addc_t* q = (const addc_t*)b;
    for (int k = 0; k < 3; k++)
        if (p->v[k] != q->v[k]) return p->v[k] < q->v[k] ? -1 : 1;
    return 0;
}

/* Adds N_add = min(floor(fac_add N_current), N_total - N_current) points
 * (at least one, at most one per valid triangle) at the centroids of the
 * valid triangles with the largest R_circ / h_i, where R_circ is the
 * circumradius and h_i the desired edge length of the geometry cell holding
 * the centroid (Sec. 3.6).  Ties in the ratio go to the smaller ascending
 * vertex triple.  The new points take the indices N_current,
 * N_current + 1, ... in the ascending order of their triangles' vertex
 * triples.  Then h_i, geps_i and h_avg are multiplied by
 * sqrt(N_old / N_current) (Sec. 3.7), and each new point is classified
 * like an initial point with the rescaled quantities (inner, else boundary)
 * and starts with a previous move of h_i.  Returns N_add. */
static int64_t add_points(om_mesh* m) {
    int64_t N0 = m->N;
    int64_t nadd = (int64_t)floor(m->P.fac_add * (double)N0);
    if (nadd < 1) nadd = 1;
    if (nadd > m->Ntot - N0) nadd = m->Ntot - N0;
    if (nadd > m->ntri) nadd = m->ntri;
    if (nadd <= 0) return 0;
    addc_t* c = (addc_t*)malloc(sizeof(addc_t) * (size_t)m->ntri);
    if (!c) return 0;
    for (int64_t t = 0; t < m->ntri; t++) {
        int32_t i = m->tri[3 * t], j = m->tri[3 * t + 1], k = m->tri[3 * t + 2]; /* i smallest, CCW */
        double ox, oy, R;
        circumcenter_fixed(m->x[i], m->y[i], m->x[j], m->y[j], m->x[k], m->y[k], &ox, &oy, &R);
        double gx = ((m->x[i] + m->x[j]) + m->x[k]) / 3.0;
        double gy = ((m->y[i] + m->y[j]) + m->y[k]) / 3.0;
        double r = R / h_at(m, gx, gy);
        c[t].ratio = r > 0.0 ? r : 0.0; /* a NaN ratio ranks last */
        c[t].v[0] = i;
        c[t].v[1] = j < k ? j : k;
        c[t].v[2] = j < k ? k : j;
        c[t].gx = gx;
        c[t].gy = gy;
    }
    qsort(c, (size_t)m->ntri, sizeof(addc_t), addc_rank_cmp);
    qsort(c, (size_t)nadd, sizeof(addc_t), addc_triple_cmp);
    double s = sqrt((double)N0 / (double)(N0 + nadd));
    size_t nc = (size_t)m->ncx * (size_t)m->ncy;
    for (size_t q = 0; q < nc; q++) {
        m->gh[q] *= s;
        m->ggeps[q] *= s;
    }
    m->havg *= s;
    for (int64_t r = 0; r < nadd; r++) {
        int64_t p = N0 + r;
        m->x[p] = c[r].gx;
        m->y[p] = c[r].gy;
        m->cls[p] = classify(m, m->x[p], m->y[p]) == PT_INNER ? PT_INNER : PT_BOUNDARY;
        m->dprev[p] = h_at(m, m->x[p], m->y[p]);
        m->pnew[2 * p] = m->x[p];
        m->pnew[2 * p + 1] = m->y[p];
    }
    free(c);
    m->N = N0 + nadd;
    m->retri = 1;
    return nadd;
}

/* Procedure I, quality (Eqs. 11-12), the hybrid switch and the termination
 * tests (Sec. 4), then the raw move; returns 1 if a termination test held,
 * 2 if points were added (no move then). */
static int triangulate_and_move(om_mesh* m) {
    om_rebuild(m);
    m->st.triangulated = 1;
    for (int64_t i = 0; i < m->N; i++) { m->tx[i] = m->x[i]; m->ty[i] = m->y[i]; }
    double qa = m->st.half_mean_alpha, qb = m->st.half_mean_beta, qm = m->st.max_alpha;
    double ra = 1, rb = 1, rm = 1;
    if (m->have_prev) {
        ra = fabs(qa - m->prev_a) / m->prev_a;
        rb = fabs(qb - m->prev_b) / m->prev_b;
        rm = fabs(qm - m->prev_amax) / m->prev_amax;
    }
    int method;
    int terminated = 0;
    int quality_end = m->have_prev && ra < m->P.T_end_q && rb < m->P.T_end_q && rm < m->P.T_end_amax;
    if (m->N < m->Ntot) {
        /* Sec. 3.6: until N_total is reached, a stalled mesh gets new points;
         * the hybrid switch and the termination tests wait for N_total */
        if (m->have_prev && ra < m->P.T_add && rb < m->P.T_add && m->ntri > 0) {
            for (int64_t i = 0; i < m->N; i++) { m->pnew[2 * i] = m->x[i]; m->pnew[2 * i + 1] = m->y[i]; }
            m->st.added = add_points(m);
            m->have_prev = 0; /* the next change is not measured across the addition */
            m->st.method_used = -1;
            m->st.switched = m->switched;
            m->st.terminated = 0;
            return 2;
        }
        method = m->P.method == 1 ? 1 : 0;
    } else if (m->P.method == 2) {
        if (!m->switched) {
            if (m->have_prev && ra < m->P.T_switch) m->switched = 1; /* Sec. 4.2: switch to CVD */
        } else if (quality_end) terminated = 1;
        method = m->switched ? 1 : 0;
    } else {
        method = m->P.method;
        terminated = quality_end;
    }
    m->prev_a = qa; m->prev_b = qb; m->prev_amax = qm; m->have_prev = 1;
    m->st.method_used = method;
    m->st.switched = m->switched;
    m->st.terminated = terminated;
    if (terminated) {
        for (int64_t i = 0; i < m->N; i++) { m->pnew[2 * i] = m->x[i]; m->pnew[2 * i + 1] = m->y[i]; }
        return 1;
    }
    if (method == 0) distmesh_move(m); else cvd_move(m);
    return 0;
}

/* Algorithm 1 (DistMesh): re-triangulate only when some point moved more
 * than fac_retria h_i (h at its cell when triangulated) since the last
 * triangulation; otherwise the springs act along the last triangulation's
 * valid edges at the current positions (fac_mu from Eq. 3 at those
 * positions), and neither quality nor the termination tests are evaluated. */
int om_step(om_mesh* m) {
    m->st.newton_fail = m->st.trace_cap = m->st.quad_cap = 0;
    m->st.small_moves = 0;
    m->st.added = 0;
    if (m->P.method == 0 && m->P.fac_retria > 0 && !m->retri) {
        fac_mu_current(m);
        m->st.method_used = 0;
        m->st.triangulated = 0;
        m->st.terminated = 0;
        distmesh_move(m);
    } else {
        int r = triangulate_and_move(m);
        if (r) {
            m->st.n_points = m->N;
            return r;
        }
    }
    int small = 1, far = 0;
    int64_t nfail = 0, tcap = 0;
#pragma omp parallel for num_threads(m->threads > 1 ? m->threads : 1) schedule(static) \
    reduction(&& : small) reduction(|| : far) reduction(+ : nfail, tcap)
    for (int64_t i = 0; i < m->N; i++) {
        double po[2] = {m->x[i], m->y[i]}, pf[2];
        int32_t nc;
        int oc = m->cls[i];
        treat_point(m, po, oc, m->pnew + 2 * i, pf, &nc, &nfail, &tcap);
        double mv = hypot(pf[0] - po[0], pf[1] - po[1]);
        if (oc == PT_INNER && !(mv < m->P.fac_end * h_at(m, po[0], po[1]))) small = 0;
        if (m->P.fac_retria > 0 && hypot(pf[0] - m->tx[i], pf[1] - m->ty[i]) > m->P.fac_retria * h_at(m, m->tx[i], m->ty[i]))
            far = 1;
        m->dprev[i] = mv;
        m->x[i] = pf[0];
        m->y[i] = pf[1];
        m->cls[i] = (uint8_t)nc;
    }
    m->st.newton_fail += nfail;
    m->st.trace_cap += tcap;
    m->st.small_moves = small;
    m->st.n_points = m->N;
    m->retri = m->P.method != 0 || !(m->P.fac_retria > 0) || far;
    return 0;
}

/* Per-cell work of one iteration on a subset of cells, for timing: the
 * cell (Sec. 2.1), its owned triangles with Tests 1-3 (Sec. 4.1) and, with
 * with_centroid, its CVD centroid (Sec. 4.2).  Returns the triangles kept. */
/* Procedure I restricted to the given cells: each cell's clip, the valid
 * triangles it owns (smallest index first, counter-clockwise) and, with
 * with_centroid, its CVD centroid.  Owned triangles are written to tri (up to
 * cap of them) when tri is not NULL; returns how many there are. */
static int64_t sample_cells(om_mesh* m, const int64_t* cells, int64_t ncells, int with_centroid, int32_t* tri,
                            int64_t cap) {
    ogrid_t G;
    ogrid_build(m, &G);
    hp_t E[CELL_CAP];
    int32_t lab[CELL_CAP];
    double poly[2 * CELL_CAP];
    int64_t errs = 0;
    int64_t kept = 0;
    for (int64_t q = 0; q < ncells; q++) {
        int64_t i = cells[q];
        int ne = cell_compute(m, &G, i, E, &errs);
        for (int t = 0; t < ne; t++) lab[t] = E[t].lab;
        for (int t = 0; t < ne; t++) {
            int32_t j = lab[t], k = lab[(t + 1) % ne];
            if (j < 0 || k < 0 || !(i < j && i < k)) continue;
            double ox, oy, R;
            circumcenter_fixed(m->x[i], m->y[i], m->x[j], m->y[j], m->x[k], m->y[k], &ox, &oy, &R);
            if (!(reg_contains(m, i, ox, oy) && reg_contains(m, j, ox, oy) && reg_contains(m, k, ox, oy))) continue;
            if (m->P.validity && !triangle_valid(m, i, j, k)) continue;
            if (tri && kept < cap) {
                tri[3 * kept] = (int32_t)i;
                tri[3 * kept + 1] = j;
                tri[3 * kept + 2] = k;
            }
            kept++;
        }
        if (with_centroid) {
            int n = cell_polygon_labels(m, i, lab, ne, poly, CELL_CAP);
            double gen[2] = {m->x[i], m->y[i]}, c[2];
            double h = h_at(m, m->x[i], m->y[i]);
            int32_t lv;
            if (n >= 3)
                centroid_adaptive(&m->siz, gen, poly, n, fmax(m->dprev[i] / h, m->P.fac_end), m->P.quad_max_level,
                                  c, &lv, NULL);
        }
    }
    ogrid_free(&G);
    return kept;
}

int om_rebuild_sample(om_mesh* m, const int64_t* cells, int64_t ncells, int with_centroid) {
    return (int)sample_cells(m, cells, ncells, with_centroid, NULL, 0);
}

/* The same work spread over nthreads OpenMP threads (cells are independent);
 * only for timing the oracle on all host cores.  Returns the number of owned
 * valid triangles. */
int64_t om_rebuild_sample_mt(om_mesh* m, const int64_t* cells, int64_t ncells, int with_centroid, int nthreads) {
    ogrid_t G;
    ogrid_build(m, &G);
    int64_t kept = 0;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 256) reduction(+ : kept)
    for (int64_t q = 0; q < ncells; q++) {
        hp_t E[CELL_CAP];
        int32_t lab[CELL_CAP];
        double poly[2 * CELL_CAP];
        int64_t errs = 0;
        int64_t i = cells[q];
        int ne = cell_compute(m, &G, i, E, &errs);
        for (int t = 0; t < ne; t++) lab[t] = E[t].lab;
        for (int t = 0; t < ne; t++) {
            int32_t j = lab[t], k = lab[(t + 1) % ne];
            if (j < 0 || k < 0 || !(i < j && i < k)) continue;
            double ox, oy, R;
            circumcenter_fixed(m->x[i], m->y[i], m->x[j], m->y[j], m->x[k], m->y[k], &ox, &oy, &R);
            if (!(reg_contains(m, i, ox, oy) && reg_contains(m, j, ox, oy) && reg_contains(m, k, ox, oy))) continue;
            if (m->P.validity && !triangle_valid(m, i, j, k)) continue;
            kept++;
        }
        if (with_centroid) {
            int n = cell_polygon_labels(m, i, lab, ne, poly, CELL_CAP);
            double gen[2] = {m->x[i], m->y[i]}, c[2];
            double h = h_at(m, m->x[i], m->y[i]);
            int32_t lv;
            if (n >= 3)
                centroid_adaptive(&m->siz, gen, poly, n, fmax(m->dprev[i] / h, m->P.fac_end), m->P.quad_max_level,
                                  c, &lv, NULL);
        }
    }
    ogrid_free(&G);
    return kept;
}

int64_t om_sample_triangles(om_mesh* m, const int64_t* cells, int64_t ncells, int32_t* tri, int64_t cap) {
    return sample_cells(m, cells, ncells, 0, tri, cap);
}

/* ------------------------------------------------------------------------ */
/* accessors                                                                */
/* ------------------------------------------------------------------------ */
int64_t om_num_points(const om_mesh* m) { return m->N; }
void om_set_threads(om_mesh* m, int threads) { m->threads = threads > 1 ? threads : 1; }
int64_t om_num_triangles(const om_mesh* m) { return m->ntri; }
void om_get_triangles(const om_mesh* m, int32_t* tri) { memcpy(tri, m->tri, sizeof(int32_t) * 3 * (size_t)m->ntri); }
int64_t om_num_edges(const om_mesh* m) { return m->nedge; }
void om_get_edges(const om_mesh* m, int32_t* e) { memcpy(e, m->edge, sizeof(int32_t) * 2 * (size_t)m->nedge); }
void om_get_points(const om_mesh* m, double* xy) {
    for (int64_t i = 0; i < m->N; i++) { xy[2 * i] = m->x[i]; xy[2 * i + 1] = m->y[i]; }
}
void om_set_points(om_mesh* m, const double* xy) {
    for (int64_t i = 0; i < m->N; i++) { m->x[i] = xy[2 * i]; m->y[i] = xy[2 * i + 1]; }
    m->retri = 1;
}
void om_get_class(const om_mesh* m, uint8_t* c) { memcpy(c, m->cls, (size_t)m->N); }
void om_set_class(om_mesh* m, const uint8_t* c) { memcpy(m->cls, c, (size_t)m->N); }
void om_get_dprev(const om_mesh* m, double* d) { memcpy(d, m->dprev, sizeof(double) * (size_t)m->N); }
void om_set_dprev(om_mesh* m, const double* d) { memcpy(m->dprev, d, sizeof(double) * (size_t)m->N); }
void om_set_method_state(om_mesh* m, int32_t switched, double pa, double pb, double pm) {
    m->switched = switched;
    m->have_prev = pa > 0;
    m->prev_a = pa; m->prev_b = pb; m->prev_amax = pm;
}
void om_get_pnew(const om_mesh* m, double* xy) { memcpy(xy, m->pnew, sizeof(double) * 2 * (size_t)m->N); }
void om_get_force(const om_mesh* m, double* f) { memcpy(f, m->force, sizeof(double) * 2 * (size_t)m->N); }
void om_get_fsum(const om_mesh* m, double* s) { memcpy(s, m->fsum, sizeof(double) * (size_t)m->N); }
void om_get_centroid(const om_mesh* m, double* c) { memcpy(c, m->cen, sizeof(double) * 2 * (size_t)m->N); }
void om_get_cell_area(const om_mesh* m, double* a) { memcpy(a, m->area, sizeof(double) * (size_t)m->N); }
void om_get_quad_level(const om_mesh* m, int32_t* lv) { memcpy(lv, m->qlevel, sizeof(int32_t) * (size_t)m->N); }
void om_get_stats(const om_mesh* m, om_stats* s) {
    *s = m->st;
    s->n_points = m->N;
}

/* ------------------------------------------------------------------------ */
/* quality report (Sec. 3.6 Eqs. 11-12; the statistics of the Sec. 5 tables) */
/* ------------------------------------------------------------------------ */
static int dbl_cmp(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

void om_quality_report(const om_mesh* m, om_quality* q) {
    static const double edge[10] = {1.0, 1.05, 1.1, 1.2, 1.3, 1.5, 2.0, 3.0, 5.0, 10.0};
    memset(q, 0, sizeof *q);
    int64_t n = m->ntri, ne = m->nedge;
    q->n_tri = n;
    q->n_edges = ne;
    q->fac_mu = m->st.fac_mu;
    double* al = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* be = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double minang = 180.0;
    for (int64_t t = 0; t < n; t++) {
        int32_t a = m->tri[3 * t], b = m->tri[3 * t + 1], c = m->tri[3 * t + 2];
        double la = hypot(m->x[b] - m->x[c], m->y[b] - m->y[c]);
        double lb = hypot(m->x[c] - m->x[a], m->y[c] - m->y[a]);
        double lc = hypot(m->x[a] - m->x[b], m->y[a] - m->y[b]);
        double o = (m->x[b] - m->x[a]) * (m->y[c] - m->y[a]) - (m->y[b] - m->y[a]) * (m->x[c] - m->x[a]);
        double A = 0.5 * fabs(o);
        al[t] = (la * lb * lc * (la + lb + lc)) / (16.0 * A * A);
        double lmax = fmax(la, fmax(lb, lc)), lmin = fmin(la, fmin(lb, lc));
        be[t] = lmax / lmin;
        double p, r;
        if (lmin == la) { p = lb; r = lc; } else if (lmin == lb) { p = la; r = lc; } else { p = la; r = lb; }
        double cs = (p * p + r * r - lmin * lmin) / (2.0 * p * r);
        if (cs > 1.0) cs = 1.0;
        if (cs < -1.0) cs = -1.0;
        double ang = acos(cs) * (180.0 / M_PI);
        if (ang < minang) minang = ang;
    }
    if (n > 0) {
        double sa = 0, sb = 0;
        for (int64_t t = 0; t < n; t++) { sa += al[t]; sb += be[t]; }
        q->mean_alpha = sa / (double)n;
        q->mean_beta = sb / (double)n;
        double va = 0, vb = 0;
        int64_t lt12 = 0, lt2 = 0;
        for (int64_t t = 0; t < n; t++) {
            va += (al[t] - q->mean_alpha) * (al[t] - q->mean_alpha);
            vb += (be[t] - q->mean_beta) * (be[t] - q->mean_beta);
            if (al[t] < 1.2) lt12++;
            if (al[t] < 2.0) lt2++;
            int k = 0;
            while (k < 9 && al[t] >= edge[k + 1]) k++;
            q->alpha_hist[k]++;
            if (al[t] > q->max_alpha) q->max_alpha = al[t];
            if (be[t] > q->max_beta) q->max_beta = be[t];
        }
        q->std_alpha = sqrt(va / (double)n);
        q->std_beta = sqrt(vb / (double)n);
        q->frac_alpha_lt_1_2 = (double)lt12 / (double)n;
        q->frac_alpha_lt_2 = (double)lt2 / (double)n;
        q->min_angle_deg = minang;
        qsort(al, (size_t)n, sizeof(double), dbl_cmp);
        qsort(be, (size_t)n, sizeof(double), dbl_cmp);
        q->median_alpha = al[(n - 1) / 2];
        q->median_beta = be[(n - 1) / 2];
    }
    free(al);
    free(be);
    if (ne > 0) {
        double* dv = (double*)malloc(sizeof(double) * (size_t)ne);
        double sd = 0;
        for (int64_t e = 0; e < ne; e++) {
            int32_t i = m->edge[2 * e], j = m->edge[2 * e + 1];
            double dx = m->x[j] - m->x[i], dy = m->y[j] - m->y[i];
            double mu = bilin(&m->siz, (m->x[i] + m->x[j]) * 0.5, (m->y[i] + m->y[j]) * 0.5);
            dv[e] = fabs(sqrt(dx * dx + dy * dy) / (q->fac_mu * mu) - 1.0);
            sd += dv[e];
        }
        q->mean_size_dev = sd / (double)ne;
        qsort(dv, (size_t)ne, sizeof(double), dbl_cmp);
        int64_t r = (int64_t)ceil(0.95 * (double)ne) - 1;
        q->p95_size_dev = dv[r < 0 ? 0 : r];
        free(dv);
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: SDF from clockwise line segments (brute force)                 */
/* ------------------------------------------------------------------------ */
static void seg_normal(const double* xy, int64_t nv, int64_t k, double* nx, double* ny) {
    int64_t k1 = k + 1 == nv ? 0 : k + 1;
    double dx = xy[2 * k1] - xy[2 * k], dy = xy[2 * k1 + 1] - xy[2 * k + 1];
    double L = sqrt(dx * dx + dy * dy);
    *nx = dy / L; /* right of the direction: inward for a clockwise loop */
    *ny = -dx / L;
}

int om_segment_sdf(const double* xy, int64_t nv, const double* px, const double* py, int64_t np, double* out) {
    if (nv < 3 || !xy || (np > 0 && (!px || !py || !out))) { set_err("bad segment input"); return -1; }
    for (int64_t q = 0; q < np; q++) {
        double x = px[q], y = py[q];
        double best = INFINITY, bt = 0.0;
        int64_t bk = -1;
        for (int64_t k = 0; k < nv; k++) {
            int64_t k1 = k + 1 == nv ? 0 : k + 1;
            double ax = xy[2 * k], ay = xy[2 * k + 1];
            double ex = xy[2 * k1] - ax, ey = xy[2 * k1 + 1] - ay;
            double wx = x - ax, wy = y - ay;
            double t = (wx * ex + wy * ey) / (ex * ex + ey * ey);
            if (!(t > 0.0)) t = 0.0;
            if (t > 1.0) t = 1.0;
            double cx = ax + t * ex, cy = ay + t * ey;
            double dx = x - cx, dy = y - cy;
            double d = sqrt(dx * dx + dy * dy);
            if (d < best) { best = d; bk = k; bt = t; }
        }
        int64_t k1 = bk + 1 == nv ? 0 : bk + 1;
        double ax = xy[2 * bk], ay = xy[2 * bk + 1];
        double ex = xy[2 * k1] - ax, ey = xy[2 * k1 + 1] - ay;
        double cx = ax + bt * ex, cy = ay + bt * ey;
        double nx, ny;
        seg_normal(xy, nv, bk, &nx, &ny);
        if (bt == 0.0 || bt == 1.0) {
            /* an end point: the sum of the incident segments' unit normals */
            int64_t other = bt == 0.0 ? (bk == 0 ? nv - 1 : bk - 1) : k1;
            double mx, my;
            seg_normal(xy, nv, other, &mx, &my);
            nx += mx;
            ny += my;
        }
        double s = (x - cx) * nx + (y - cy) * ny;
        out[q] = s > 0.0 ? -best : best;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.7: adaptive distance field on boundary grid cells                 */
/* ------------------------------------------------------------------------ */
struct om_adf {
    double x0, y0, dx, dy;
    int32_t ncx, ncy, ncells;
    int32_t* cells;
    int32_t* cellroot; /* [ncx * ncy] tree of each cell or -1 */
    int64_t n, cap;
    double* v;
    int32_t *child, *root, *lev;
};

static int adf_grow(om_adf* a, int64_t need) {
    if (need <= a->cap) return 0;
    int64_t cap = a->cap ? a->cap : 1024;
    while (cap < need) cap *= 2;
    double* v = (double*)realloc(a->v, sizeof(double) * 4 * (size_t)cap);
    if (v) a->v = v;
    int32_t* c = (int32_t*)realloc(a->child, sizeof(int32_t) * (size_t)cap);
    if (c) a->child = c;
    int32_t* r = (int32_t*)realloc(a->root, sizeof(int32_t) * (size_t)cap);
    if (r) a->root = r;
    int32_t* l = (int32_t*)realloc(a->lev, sizeof(int32_t) * 3 * (size_t)cap);
    if (l) a->lev = l;
    if (!v || !c || !r || !l) return -1;
    a->cap = cap;
    return 0;
}

/* coordinate of node corner index i at level L of a cell starting at c0 */
static double adf_coord(double c0, double w, int32_t i, int32_t L) {
    return c0 + (double)i * (w * (1.0 / (double)(1 << L)));
}

static int adf_push(om_adf* a, int32_t root, int32_t L, int32_t ix, int32_t iy, double v00, double v10, double v01,
                    double v11) {
    if (adf_grow(a, a->n + 1)) return -1;
    int64_t k = a->n++;
    a->v[4 * k] = v00;
    a->v[4 * k + 1] = v10;
    a->v[4 * k + 2] = v01;
    a->v[4 * k + 3] = v11;
    a->child[k] = -1;
    a->root[k] = root;
    a->lev[3 * k] = L;
    a->lev[3 * k + 1] = ix;
    a->lev[3 * k + 2] = iy;
    return 0;
}

void om_adf_free(om_adf* a) {
    if (!a) return;
    free(a->cells); free(a->cellroot); free(a->v); free(a->child); free(a->root); free(a->lev);
    free(a);
}

om_adf* om_adf_build(const double* xy, int64_t nv, double x0, double y0, double x1, double y1, int32_t nx, int32_t ny,
                     const int32_t* cells, const double* tol, int32_t ncells, int32_t max_depth) {
    if (!xy || nv < 3 || nx < 2 || ny < 2 || !(x1 > x0) || !(y1 > y0) || ncells < 0 || (ncells > 0 && (!cells || !tol)) ||
        max_depth < 0 || max_depth > 14) {
        set_err("bad ADF input");
        return NULL;
    }
    om_adf* a = (om_adf*)calloc(1, sizeof(om_adf));
    if (!a) { set_err("oom"); return NULL; }
    a->x0 = x0;
    a->y0 = y0;
    a->dx = (x1 - x0) / (double)(nx - 1);
    a->dy = (y1 - y0) / (double)(ny - 1);
    a->ncx = nx - 1;
    a->ncy = ny - 1;
    a->ncells = ncells;
    a->cells = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ncells > 0 ? ncells : 1));
    a->cellroot = (int32_t*)malloc(sizeof(int32_t) * (size_t)a->ncx * (size_t)a->ncy);
    if (!a->cells || !a->cellroot) { om_adf_free(a); set_err("oom"); return NULL; }
    for (int64_t c = 0; c < (int64_t)a->ncx * a->ncy; c++) a->cellroot[c] = -1;
    /* level 0: the cells themselves, corners from the exact SDF */
    for (int32_t r = 0; r < ncells; r++) {
        int32_t c = cells[r];
        if (c < 0 || c >= a->ncx * a->ncy || a->cellroot[c] >= 0) { om_adf_free(a); set_err("bad ADF cell list"); return NULL; }
        a->cells[r] = c;
        a->cellroot[c] = r;
        double cx0 = x0 + (double)(c % a->ncx) * a->dx, cy0 = y0 + (double)(c / a->ncx) * a->dy;
        double xa = adf_coord(cx0, a->dx, 0, 0), xb = adf_coord(cx0, a->dx, 1, 0);
        double ya = adf_coord(cy0, a->dy, 0, 0), yb = adf_coord(cy0, a->dy, 1, 0);
        double px[4] = {xa, xb, xa, xb}, py[4] = {ya, ya, yb, yb}, s[4];
        om_segment_sdf(xy, nv, px, py, 4, s);
        if (adf_push(a, r, 0, 0, 0, s[0], s[1], s[2], s[3])) { om_adf_free(a); set_err("oom"); return NULL; }
    }
    /* level by level: test the level's nodes in order, append the children */
    int64_t lo = 0, hi = a->n;
    for (int32_t L = 0; L < max_depth && lo < hi; L++) {
        for (int64_t k = lo; k < hi; k++) {
            int32_t r = a->root[k], ix = a->lev[3 * k + 1], iy = a->lev[3 * k + 2];
            int32_t c = a->cells[r];
            double cx0 = x0 + (double)(c % a->ncx) * a->dx, cy0 = y0 + (double)(c / a->ncx) * a->dy;
            double xa = adf_coord(cx0, a->dx, 2 * ix, L + 1), xm = adf_coord(cx0, a->dx, 2 * ix + 1, L + 1);
            double xb = adf_coord(cx0, a->dx, 2 * ix + 2, L + 1);
            double ya = adf_coord(cy0, a->dy, 2 * iy, L + 1), ym = adf_coord(cy0, a->dy, 2 * iy + 1, L + 1);
            double yb = adf_coord(cy0, a->dy, 2 * iy + 2, L + 1);
            /* exact SDF at the bottom, top, left, right midpoints and the centre */
            double px[5] = {xm, xm, xa, xb, xm}, py[5] = {ya, yb, ym, ym, ym}, s[5];
            om_segment_sdf(xy, nv, px, py, 5, s);
            double v00 = a->v[4 * k], v10 = a->v[4 * k + 1], v01 = a->v[4 * k + 2], v11 = a->v[4 * k + 3];
            double p[5] = {(v00 + v10) * 0.5, (v01 + v11) * 0.5, (v00 + v01) * 0.5, (v10 + v11) * 0.5,
                           ((v00 + v10) + (v01 + v11)) * 0.25};
            double err = 0.0;
            for (int q = 0; q < 5; q++) err = fmax(err, fabs(p[q] - s[q]));
            if (!(err > tol[r])) continue;
            a->child[k] = (int32_t)a->n;
            if (adf_push(a, r, L + 1, 2 * ix, 2 * iy, v00, s[0], s[2], s[4]) ||
                adf_push(a, r, L + 1, 2 * ix + 1, 2 * iy, s[0], v10, s[4], s[3]) ||
                adf_push(a, r, L + 1, 2 * ix, 2 * iy + 1, s[2], s[4], v01, s[1]) ||
                adf_push(a, r, L + 1, 2 * ix + 1, 2 * iy + 1, s[4], s[3], s[1], v11)) {
                om_adf_free(a);
                set_err("oom");
                return NULL;
            }
        }
        lo = hi;
        hi = a->n;
    }
    return a;
}

int64_t om_adf_size(const om_adf* a) { return a ? a->n : 0; }

void om_adf_export(const om_adf* a, double* v, int32_t* child, int32_t* root, int32_t* lev) {
    memcpy(v, a->v, sizeof(double) * 4 * (size_t)a->n);
    memcpy(child, a->child, sizeof(int32_t) * (size_t)a->n);
    memcpy(root, a->root, sizeof(int32_t) * (size_t)a->n);
    memcpy(lev, a->lev, sizeof(int32_t) * 3 * (size_t)a->n);
}

void om_adf_eval(const om_adf* a, const double* px, const double* py, int64_t np, double* out) {
    for (int64_t q = 0; q < np; q++) {
        double x = px[q], y = py[q];
        double fi = floor((x - a->x0) / a->dx), fj = floor((y - a->y0) / a->dy);
        int32_t i = !(fi >= 0.0) ? 0 : (fi > (double)(a->ncx - 1) ? a->ncx - 1 : (int32_t)fi);
        int32_t j = !(fj >= 0.0) ? 0 : (fj > (double)(a->ncy - 1) ? a->ncy - 1 : (int32_t)fj);
        int32_t r = a->cellroot[j * a->ncx + i];
        if (r < 0) { out[q] = NAN; continue; }
        double cx0 = a->x0 + (double)i * a->dx, cy0 = a->y0 + (double)j * a->dy;
        int64_t k = r;
        while (a->child[k] >= 0) {
            int32_t L = a->lev[3 * k], ix = a->lev[3 * k + 1], iy = a->lev[3 * k + 2];
            double xm = adf_coord(cx0, a->dx, 2 * ix + 1, L + 1), ym = adf_coord(cy0, a->dy, 2 * iy + 1, L + 1);
            k = a->child[k] + (y >= ym ? 2 : 0) + (x >= xm ? 1 : 0);
        }
        int32_t L = a->lev[3 * k], ix = a->lev[3 * k + 1], iy = a->lev[3 * k + 2];
        double wx = a->dx * (1.0 / (double)(1 << L)), wy = a->dy * (1.0 / (double)(1 << L));
        double fx = (x - adf_coord(cx0, a->dx, ix, L)) / wx, fy = (y - adf_coord(cy0, a->dy, iy, L)) / wy;
        fx = fx < 0.0 ? 0.0 : (fx > 1.0 ? 1.0 : fx);
        fy = fy < 0.0 ? 0.0 : (fy > 1.0 ? 1.0 : fy);
        const double* v = a->v + 4 * k;
        double va = v[0] + fx * (v[1] - v[0]), vb = v[2] + fx * (v[3] - v[2]);
        out[q] = va + fy * (vb - va);
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3 Eq. 7: sizing field from boundary samples (brute force)         */
/* ------------------------------------------------------------------------ */
int om_sizing_field(const double* sxy, const double* lfs, int64_t ns, double K, const double* px, const double* py,
                    int64_t np, double* out) {
    if (ns < 1 || !sxy || !lfs || !(K >= 0.0) || (np > 0 && (!px || !py || !out))) {
        set_err("bad sizing input");
        return -1;
    }
    for (int64_t q = 0; q < np; q++) {
        double best = INFINITY;
        for (int64_t k = 0; k < ns; k++) {
            double dx = px[q] - sxy[2 * k], dy = py[q] - sxy[2 * k + 1];
            double v = K * sqrt(dx * dx + dy * dy) + lfs[k];
            if (v < best) best = v;
        }
        out[q] = best;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* App. A: boundary samples; Sec. 3.3: medial axis and lfs                   */
/* ------------------------------------------------------------------------ */
static double seg_sdf1(const double* xy, int64_t nv, double x, double y) {
    double v;
    om_segment_sdf(xy, nv, &x, &y, 1, &v);
    return v;
}

int64_t om_boundary_samples(const double* xy, int64_t nv, double ds, double geps_hat, double* out, int64_t cap) {
    if (nv < 3 || !(ds > 0.0) || !(geps_hat >= 0.0)) { set_err("bad sample input"); return -1; }
    int64_t n = 0, ncap = nv;
    for (int64_t k = 0; k < nv; k++) {
        int64_t k1 = k + 1 == nv ? 0 : k + 1;
        double L = sqrt((xy[2 * k1] - xy[2 * k]) * (xy[2 * k1] - xy[2 * k]) +
                        (xy[2 * k1 + 1] - xy[2 * k + 1]) * (xy[2 * k1 + 1] - xy[2 * k + 1]));
        if (L > ds) ncap += (int64_t)floor(L / ds);
    }
    double* px = (double*)malloc(sizeof(double) * (size_t)ncap);
    double* py = (double*)malloc(sizeof(double) * (size_t)ncap);
    uint8_t* alive = (uint8_t*)malloc((size_t)ncap);
    uint8_t* done = (uint8_t*)malloc((size_t)ncap);
    if (!px || !py || !alive || !done) { free(px); free(py); free(alive); free(done); set_err("oom"); return -1; }
    for (int64_t k = 0; k < nv; k++) {
        int64_t k1 = k + 1 == nv ? 0 : k + 1;
        double ax = xy[2 * k], ay = xy[2 * k + 1], ex = xy[2 * k1] - ax, ey = xy[2 * k1 + 1] - ay;
        double L = sqrt(ex * ex + ey * ey);
        px[n] = ax; py[n] = ay; n++;
        if (L > ds) {
            int64_t m = (int64_t)floor(L / ds) + 1; /* intervals, each shorter than ds */
            for (int64_t q = 1; q < m; q++) {
                double t = (double)q / (double)m;
                px[n] = ax + t * ex; py[n] = ay + t * ey; n++;
            }
        }
    }
    for (int64_t i = 0; i < n; i++) { alive[i] = 1; done[i] = 0; }
    int any = 1;
    while (any) {
        any = 0;
        for (int64_t i = 0; i < n; i++) {
            if (!alive[i] || done[i]) continue;
            /* closest valid other point: by (distance, index) */
            double last_d = -1.0;
            int64_t last_j = -1, found = -1;
            double fd = 0.0, mx = 0.0, my = 0.0;
            for (;;) {
                double bd = INFINITY;
                int64_t bj = -1;
                for (int64_t j = 0; j < n; j++) {
                    if (j == i || !alive[j]) continue;
                    double dx = px[j] - px[i], dy = py[j] - py[i];
                    double d = sqrt(dx * dx + dy * dy);
                    /* next in (d, j) order after (last_d, last_j) */
                    if (d < last_d || (d == last_d && j <= last_j)) continue;
                    if (d < bd || (d == bd && j < bj)) { bd = d; bj = j; }
                }
                if (bj < 0) break;
                double cx = (px[i] + px[bj]) * 0.5, cy = (py[i] + py[bj]) * 0.5;
                if (fabs(seg_sdf1(xy, nv, cx, cy)) <= geps_hat) { found = bj; fd = bd; mx = cx; my = cy; break; }
                last_d = bd; last_j = bj;
            }
            if (found < 0 || !(fd < ds)) { done[i] = 1; continue; }
            alive[found] = 0;
            px[i] = mx; py[i] = my;
            any = 1;
        }
    }
    int64_t c = 0;
    for (int64_t i = 0; i < n; i++)
        if (alive[i]) {
            if (c < cap && out) { out[2 * c] = px[i]; out[2 * c + 1] = py[i]; }
            c++;
        }
    free(px); free(py); free(alive); free(done);
    return c;
}

static int triple_less(const int32_t* a, const int32_t* b) {
    int32_t x[3] = {a[0], a[1], a[2]}, y[3] = {b[0], b[1], b[2]};
    /* sort each ascending */
    for (int r = 0; r < 2; r++)
        for (int q = 0; q < 2 - r; q++) {
            if (x[q] > x[q + 1]) { int32_t t = x[q]; x[q] = x[q + 1]; x[q + 1] = t; }
            if (y[q] > y[q + 1]) { int32_t t = y[q]; y[q] = y[q + 1]; y[q + 1] = t; }
        }
    for (int q = 0; q < 3; q++)
        if (x[q] != y[q]) return x[q] < y[q];
    return 0;
}

void om_medial_points(const om_mesh* m, double* v, uint8_t* flags) {
    int64_t N = m->N;
    double* best1 = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    int64_t* t1 = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    double* cc = (double*)malloc(sizeof(double) * 2 * (size_t)(m->ntri > 0 ? m->ntri : 1));
    for (int64_t i = 0; i < N; i++) { best1[i] = -1.0; t1[i] = -1; flags[i] = 0; }
    for (int64_t t = 0; t < m->ntri; t++) {
        const int32_t* T = m->tri + 3 * t;
        double ox, oy, R;
        circumcenter_fixed(m->x[T[0]], m->y[T[0]], m->x[T[1]], m->y[T[1]], m->x[T[2]], m->y[T[2]], &ox, &oy, &R);
        cc[2 * t] = ox; cc[2 * t + 1] = oy;
        for (int q = 0; q < 3; q++) {
            int32_t p = T[q];
            double dx = ox - m->x[p], dy = oy - m->y[p];
            double d = sqrt(dx * dx + dy * dy);
            if (d > best1[p] || (d == best1[p] && t1[p] >= 0 && triple_less(T, m->tri + 3 * t1[p]))) {
                best1[p] = d; t1[p] = t;
            }
        }
    }
    for (int64_t i = 0; i < N; i++)
        if (t1[i] >= 0) { v[4 * i] = cc[2 * t1[i]]; v[4 * i + 1] = cc[2 * t1[i] + 1]; flags[i] |= 1; }
    double* best2 = best1;
    int64_t* t2 = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; i++) { best2[i] = -1.0; t2[i] = -1; }
    for (int64_t t = 0; t < m->ntri; t++) {
        const int32_t* T = m->tri + 3 * t;
        double ox = cc[2 * t], oy = cc[2 * t + 1];
        for (int q = 0; q < 3; q++) {
            int32_t p = T[q];
            if (!(flags[p] & 1)) continue;
            double ux = v[4 * p] - m->x[p], uy = v[4 * p + 1] - m->y[p];
            double dx = ox - m->x[p], dy = oy - m->y[p];
            if (!(dx * ux + dy * uy <= 0.0)) continue;
            double d = sqrt(dx * dx + dy * dy);
            if (d > best2[p] || (d == best2[p] && t2[p] >= 0 && triple_less(T, m->tri + 3 * t2[p]))) {
                best2[p] = d; t2[p] = t;
            }
        }
    }
    for (int64_t i = 0; i < N; i++)
        if (t2[i] >= 0) { v[4 * i + 2] = cc[2 * t2[i]]; v[4 * i + 3] = cc[2 * t2[i] + 1]; flags[i] |= 2; }
    free(best1); free(t1); free(t2); free(cc);
}

int64_t om_lfs(const double* sxy, int64_t ns, const double* mxy, int64_t nm, double r_nei, int32_t n_thres,
               double* lfs) {
    if (ns < 1 || nm < 1) { set_err("no samples or no medial points"); return -1; }
    uint8_t* keep = (uint8_t*)malloc((size_t)nm);
    int64_t kept = 0;
    for (int64_t a = 0; a < nm; a++) {
        int64_t c = 0;
        for (int64_t b = 0; b < nm; b++) {
            if (b == a) continue;
            double dx = mxy[2 * b] - mxy[2 * a], dy = mxy[2 * b + 1] - mxy[2 * a + 1];
            if (sqrt(dx * dx + dy * dy) <= r_nei) c++;
        }
        keep[a] = c >= n_thres;
        kept += keep[a];
    }
    for (int64_t i = 0; i < ns; i++) {
        double best = INFINITY;
        for (int64_t a = 0; a < nm; a++) {
            if (kept > 0 && !keep[a]) continue;
            double dx = mxy[2 * a] - sxy[2 * i], dy = mxy[2 * a + 1] - sxy[2 * i + 1];
            double d = sqrt(dx * dx + dy * dy);
            if (d < best) best = d;
        }
        lfs[i] = best;
    }
    free(keep);
    return kept;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.5: point initialisation                                            */
/* ------------------------------------------------------------------------ */
uint64_t om_splitmix64(uint64_t seed, uint64_t n) {
    uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int64_t om_init_points(const om_grid* sdf, const om_grid* sizing, int64_t n_init, uint64_t seed, const om_params* p,
                       double* out, int64_t cap) {
    if (n_init < 1) { set_err("n_init must be >= 1"); return -1; }
    om_mesh* m = (om_mesh*)calloc(1, sizeof *m);
    if (!m) return -1;
    if (p) m->P = *p; else om_default_params(&m->P);
    m->N = n_init;
    if (grid_copy(&m->sdf, sdf) || grid_copy(&m->siz, sizing) || geometry_setup(m)) {
        set_err("bad grids");
        om_destroy(m);
        return -1;
    }
    int ncx = m->ncx, ncy = m->ncy;
    size_t nc = (size_t)ncx * (size_t)ncy;
    double dx = m->sdf.dx, dy = m->sdf.dy;
    double band = m->P.eta * fmin(dx, dy);
    double* rho = (double*)malloc(nc * sizeof(double));
    uint8_t* sel = (uint8_t*)malloc(nc);
    double* carry = (double*)calloc(nc, sizeof(double));
    int64_t* cnt = (int64_t*)calloc(nc, sizeof(int64_t));
    double sum_rho = 0.0;
    for (int gj = 0; gj < ncy; gj++)
        for (int gi = 0; gi < ncx; gi++) {
            size_t c = cidx(m, gi, gj);
            const float* r0 = m->sdf.v + (size_t)gj * m->sdf.nx + gi;
            const float* r1 = r0 + m->sdf.nx;
            double sm = 0.25 * ((((double)r0[0] + (double)r0[1]) + (double)r1[0]) + (double)r1[1]);
            double mu = bilin(&m->siz, m->sdf.x0 + ((double)gi + 0.5) * dx, m->sdf.y0 + ((double)gj + 0.5) * dy);
            rho[c] = 1.0 / (mu * mu);
            sel[c] = m->gcls[c] == CLS_INNER || (m->gcls[c] == CLS_BOUNDARY && sm <= band);
            if (sel[c]) sum_rho += rho[c];
        }
    int64_t total = 0;
    for (int gj = 0; gj < ncy; gj++)
        for (int gi = 0; gi < ncx; gi++) {
            size_t c = cidx(m, gi, gj);
            if (!sel[c]) continue;
            double val = (rho[c] / sum_rho) * (double)n_init + carry[c];
            double k = floor(val + 0.5);
            if (k < 0.0) k = 0.0;
            double R = val - k;
            int nb[4][2] = {{gi + 1, gj}, {gi - 1, gj + 1}, {gi, gj + 1}, {gi + 1, gj + 1}};
            int mn = 0;
            for (int q = 0; q < 4; q++)
                if (nb[q][0] >= 0 && nb[q][0] < ncx && nb[q][1] < ncy && sel[cidx(m, nb[q][0], nb[q][1])]) mn++;
            for (int q = 0; q < 4 && mn > 0; q++)
                if (nb[q][0] >= 0 && nb[q][0] < ncx && nb[q][1] < ncy && sel[cidx(m, nb[q][0], nb[q][1])])
                    carry[cidx(m, nb[q][0], nb[q][1])] += R / (double)mn;
            cnt[c] = (int64_t)k;
            total += cnt[c];
        }
    int64_t g = 0;
    for (int gj = 0; gj < ncy; gj++)
        for (int gi = 0; gi < ncx; gi++) {
            size_t c = cidx(m, gi, gj);
            for (int64_t k = 0; k < cnt[c]; k++, g++) {
                double u = (double)(om_splitmix64(seed, (uint64_t)(2 * g)) >> 11) * 0x1.0p-53;
                double w = (double)(om_splitmix64(seed, (uint64_t)(2 * g + 1)) >> 11) * 0x1.0p-53;
                double cx0 = m->sdf.x0 + (double)gi * dx, cy0 = m->sdf.y0 + (double)gj * dy;
                double pt[2] = {cx0 + u * dx, cy0 + w * dy};
                if (m->gcls[c] == CLS_BOUNDARY && bilin(&m->sdf, pt[0], pt[1]) > m->ggeps[c]) {
                    /* the projection counts only when it ends as a boundary
                     * point (Sec. 4.3); otherwise the point stays where drawn */
                    double q[2];
                    newton_project(m, pt, q);
                    if (classify(m, q[0], q[1]) == PT_BOUNDARY) {
                        pt[0] = q[0];
                        pt[1] = q[1];
                    }
                }
                if (g < cap && out) { out[2 * g] = pt[0]; out[2 * g + 1] = pt[1]; }
            }
        }
    free(rho); free(sel); free(carry); free(cnt);
    om_destroy(m);
    return total;
}
