/*
 * FP64 CPU oracle for the SPH hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this code; the CUDA library neither calls it nor shares code with it.
 * It is deliberately plain: every sum runs over the neighbour set in ascending
 * particle index, in FP64, so that a reader can check it against the paper.
 *
 * Paper anchors (arXiv 2512.05516):
 *   Eq. 1-2   SPH interpolant and gradient with a compactly supported kernel W
 *   Eq. 6     density  rho_i = sum_j m_j W(r_i - r_j, h_ij)
 *   Eq. 7     momentum dv_i/dt = -sum_j m_j (P_i/rho_i^2 + P_j/rho_j^2) grad W + f_visc
 *   Eq. 5     internal energy du/dt = (P/rho^2) drho/dt + Phi
 *   Sec. 2    "the number of neighbours ... is kept approximately constant by
 *             adapting h"; cubic-spline kernels named
 *   Table 2   storage formats: IEEE single / half, and truncated single
 *   Sec. 3.2  truncated values form a packed N-bit SoA bitstream
 *
 * Readings where the paper is silent (each one is restated where it is used):
 *   R1  W is the M4 cubic spline with support 2h, sigma = 1/pi in 3D.
 *   R2  "neighbour" means r^2 < (2h)^2, strict; the self term is part of rho
 *       but not of the neighbour count.
 *   R3  the density uses the gather form h_ij = h_i (needed by the h iteration).
 *   R4  sums run over j in ascending original index.
 *   R5  h iteration: exactly `newton_steps` Newton steps on
 *       f(h) = rho(h) - m_i (eta/h)^3, each step clamped to [h/2, 2h] and to
 *       h <= h_cap, followed by one more density sum at the final h.
 *   R6  ideal gas: P = (gamma-1) rho u, c = sqrt(gamma P / rho).
 *   R7  the force uses h_ij = (h_i + h_j)/2 and a pair interacts iff r < 2 h_ij.
 *   R8  f_visc is Monaghan's artificial viscosity with alpha, beta, eps.
 *   R9  no grad-h terms, no external force.
 *   R10 kick/drift: v += a dt, u += du/dt dt, x += v dt, then periodic wrap.
 *   R11 FP64 -> FP32 is IEEE round-to-nearest-even; half and bfloat16 are
 *       rounded to nearest even from that FP32 value; the truncated formats keep
 *       sign, 8 exponent bits and the top N mantissa bits (truncation toward 0).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* R1: 3D normalisation of the M4 spline whose support is 2h. */
#define SIGMA3 (1.0 / M_PI)

/* ------------------------------------------------------------------------- */
/* Smoothing kernel (R1)                                                      */
/* ------------------------------------------------------------------------- */

/* dimensionless spline w(q), q = r/h */
double orc_w(double q)
{
    if (q < 0.0) q = -q;
    if (q < 1.0) return 1.0 - 1.5 * q * q + 0.75 * q * q * q;
    if (q < 2.0) { double t = 2.0 - q; return 0.25 * t * t * t; }
    return 0.0;
}

/* dw/dq */
double orc_dw(double q)
{
    if (q < 1.0) return -3.0 * q + 2.25 * q * q;
    if (q < 2.0) { double t = 2.0 - q; return -0.75 * t * t; }
    return 0.0;
}

/* W(r, h) = sigma / h^3 * w(r/h) */
double orc_W(double r, double h)
{
    return SIGMA3 / (h * h * h) * orc_w(r / h);
}

/* dW/dr = sigma / h^4 * w'(r/h) */
double orc_dWdr(double r, double h)
{
    return SIGMA3 / (h * h * h * h) * orc_dw(r / h);
}

/* dW/dh = -sigma / h^4 * (3 w(q) + q w'(q)) */
double orc_dWdh(double r, double h)
{
    double q = r / h;
    return -SIGMA3 / (h * h * h * h) * (3.0 * orc_w(q) + q * orc_dw(q));
}

/* ------------------------------------------------------------------------- */
/* Periodic geometry                                                          */
/* ------------------------------------------------------------------------- */

/* minimum-image separation d = x_i - x_j in a periodic box */
static void min_image(const double *xi, const double *xj, const double *box, double *d)
{
    for (int k = 0; k < 3; ++k) {
        double t = xi[k] - xj[k];
        t -= box[k] * nearbyint(t / box[k]);
        d[k] = t;
    }
}

static double norm2(const double *d)
{
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

/* cell coordinate along one axis: floor(x * (nc / L)), clamped to [0, nc-1] */
static int32_t cell_coord(double x, double inv, int32_t nc)
{
    double f = floor(x * inv);
    if (!(f >= 0.0)) return 0;            /* also catches NaN */
    if (f > (double)(nc - 1)) return nc - 1;
    return (int32_t)f;
}

/* ------------------------------------------------------------------------- */
/* Binning: FP64 cell index, stable counting sort                             */
/* ------------------------------------------------------------------------- */

/*
 * Cells with sub-cells: each of the nc_x nc_y nc_z cells is split into
 * sub^3 sub-cells.  Fine coordinate f_d = clamp(floor(x_d * (sub nc_d / L_d)),
 * 0, sub nc_d - 1); cell k_d = f_d / sub, sub-cell s_d = f_d % sub; key
 * (kx + nc_x (ky + nc_y kz)) sub^3 + (s_x + sub (s_y + sub s_z)).  perm lists
 * the particles by key, ascending original index among equal keys;
 * cell_start[key] is the first slot of that sub-cell, cell_start[ncell sub^3]
 * = n.  With sub = 1 this is the plain cell list.  Returns 0, or -1 on a bad
 * grid.
 */
int orc_bin_sub(int64_t n, const double *x, const double *box, const int32_t *nc, int32_t sub,
                int32_t *cell_of, int64_t *perm, int64_t *cell_start)
{
    if (nc[0] < 1 || nc[1] < 1 || nc[2] < 1 || sub < 1) return -1;
    const int64_t s3 = (int64_t)sub * sub * sub;
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2] * s3;
    double inv[3];
    int32_t nf[3];
    for (int k = 0; k < 3; ++k) {
        nf[k] = nc[k] * sub;
        inv[k] = (double)nf[k] / box[k];
    }
    for (int64_t c = 0; c <= ncell; ++c) cell_start[c] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t f[3], k[3], s[3];
        for (int a = 0; a < 3; ++a) {
            f[a] = cell_coord(x[3 * i + a], inv[a], nf[a]);
            k[a] = f[a] / sub;
            s[a] = f[a] % sub;
        }
        int64_t cell = k[0] + (int64_t)nc[0] * (k[1] + (int64_t)nc[1] * k[2]);
        int32_t c = (int32_t)(cell * s3 + (s[0] + sub * (s[1] + sub * s[2])));
        cell_of[i] = c;
        cell_start[c + 1] += 1;
    }
    for (int64_t c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncell > 0 ? ncell : 1));
    if (!fill) return -1;
    for (int64_t c = 0; c < ncell; ++c) fill[c] = cell_start[c];
    for (int64_t i = 0; i < n; ++i) perm[fill[cell_of[i]]++] = i;
    free(fill);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Level hierarchy for per-particle h: Morton keys of the finest cells        */
/* ------------------------------------------------------------------------- */

/* Morton (Z-order) code, written bit by bit: bit b of fx, fy, fz goes to bit
 * 3b, 3b + 1, 3b + 2 of the key */
static int64_t morton3(int32_t fx, int32_t fy, int32_t fz, int bits)
{
    int64_t k = 0;
    for (int b = 0; b < bits; ++b) {
        k |= (int64_t)((fx >> b) & 1) << (3 * b);
        k |= (int64_t)((fy >> b) & 1) << (3 * b + 1);
        k |= (int64_t)((fz >> b) & 1) << (3 * b + 2);
    }
    return k;
}

typedef struct { int64_t key, idx; } keyidx_t;

static int cmp_keyidx(const void *pa, const void *pb)
{
    const keyidx_t *a = (const keyidx_t *)pa, *b = (const keyidx_t *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

/*
 * Section 2 gives every particle its own h (adapted to a fixed neighbour
 * number); the paper's SWIFT kernels search neighbours in a cell tree.  This
 * is the hierarchy read from that, as a linear octree:
 * levels l = level_min..level_max: 2^l cells per axis, edge L_d / 2^l.  The
 * key of a particle is the Morton code of its finest cell, f_d =
 * clamp(floor(x_d * (2^level_max / L_d)), 0, 2^level_max - 1).  Its level is
 * the largest l with h (1 + margin) <= h_l = min_d (L_d / 2^l) / 2, or
 * level_min when no level qualifies or h is not finite and positive.  perm
 * lists the particles by key, ascending index among equal keys.  Returns 0,
 * or -1 on bad levels.
 */
int orc_levels(int64_t n, const double *x, const double *h, const double *box, int32_t level_min,
               int32_t level_max, double margin, int32_t *key, int8_t *level, int64_t *perm)
{
    if (level_min < 0 || level_max > 20 || level_min > level_max) return -1;
    const int32_t F = (int32_t)1 << level_max;
    const double grow = 1.0 + margin;
    keyidx_t *ki = (keyidx_t *)malloc(sizeof(keyidx_t) * (size_t)(n > 0 ? n : 1));
    if (!ki) return -1;
    for (int64_t i = 0; i < n; ++i) {
        int32_t f[3];
        for (int a = 0; a < 3; ++a) f[a] = cell_coord(x[3 * i + a], (double)F / box[a], F);
        const int64_t k = morton3(f[0], f[1], f[2], level_max);
        key[i] = (int32_t)k;
        ki[i].key = k;
        ki[i].idx = i;
        int lv = level_min;
        if (isfinite(h[i]) && h[i] > 0.0) {
            const double t = h[i] * grow;
            for (int l = level_max; l > level_min; --l) {
                double e = ldexp(box[0], -l);
                for (int a = 1; a < 3; ++a)
                    if (ldexp(box[a], -l) < e) e = ldexp(box[a], -l);
                if (t <= 0.5 * e) {
                    lv = l;
                    break;
                }
            }
        }
        level[i] = (int8_t)lv;
    }
    qsort(ki, (size_t)n, sizeof(keyidx_t), cmp_keyidx);
    for (int64_t s = 0; s < n; ++s) perm[s] = ki[s].idx;
    free(ki);
    return 0;
}

/* plain cell list: one sub-cell per cell */
int orc_bin(int64_t n, const double *x, const double *box, const int32_t *nc,
            int32_t *cell_of, int64_t *perm, int64_t *cell_start)
{
    return orc_bin_sub(n, x, box, nc, 1, cell_of, perm, cell_start);
}

/* ------------------------------------------------------------------------- */
/* Neighbour search support: a cell list only narrows the candidate set; the  */
/* neighbour set itself is the exact distance test, summed in ascending j.    */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t nc[3];
    double inv[3];
    int64_t ncell;
    int64_t *start;
    int64_t *idx;
    int32_t *cell_of;
} grid_t;

static int grid_build(grid_t *g, int64_t n, const double *x, const double *box, double edge)
{
    memset(g, 0, sizeof(*g));
    if (!(edge > 0.0)) return 0;
    for (int k = 0; k < 3; ++k) {
        double f = floor(box[k] / edge);
        if (f < 3.0) return 0;            /* too few cells: use brute force */
        if (f > 256.0) f = 256.0;         /* larger cells still cover the radius */
        g->nc[k] = (int32_t)f;
    }
    g->ncell = (int64_t)g->nc[0] * g->nc[1] * g->nc[2];
    g->start = (int64_t *)malloc(sizeof(int64_t) * (size_t)(g->ncell + 1));
    g->idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    g->cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!g->start || !g->idx || !g->cell_of) return 0;
    if (orc_bin(n, x, box, g->nc, g->cell_of, g->idx, g->start) != 0) return 0;
    for (int k = 0; k < 3; ++k) g->inv[k] = (double)g->nc[k] / box[k];
    return 1;
}

static void grid_free(grid_t *g)
{
    free(g->start); free(g->idx); free(g->cell_of);
    memset(g, 0, sizeof(*g));
}

typedef struct { int64_t j; double r2; double d[3]; } cand_t;

typedef struct { cand_t *c; int64_t n, cap; } cbuf_t;

static void cbuf_push(cbuf_t *b, int64_t j, const double *d, double r2)
{
    if (b->n == b->cap) {
        b->cap = b->cap ? 2 * b->cap : 4096;
        b->c = (cand_t *)realloc(b->c, sizeof(cand_t) * (size_t)b->cap);
    }
    cand_t *e = &b->c[b->n++];
    e->j = j; e->r2 = r2; e->d[0] = d[0]; e->d[1] = d[1]; e->d[2] = d[2];
}

/* All particles j that can lie within the grid edge of particle i (or all of
 * them when brute force is used), with their separation x_i - x_j. */
static void gather_candidates(cbuf_t *b, const grid_t *g, int brute, int64_t n,
                              const double *x, const double *box, int64_t i)
{
    b->n = 0;
    double d[3];
    if (brute || g->ncell == 0) {
        for (int64_t j = 0; j < n; ++j) {
            min_image(&x[3 * i], &x[3 * j], box, d);
            cbuf_push(b, j, d, norm2(d));
        }
        return;
    }
    int32_t k[3];
    for (int a = 0; a < 3; ++a) k[a] = cell_coord(x[3 * i + a], g->inv[a], g->nc[a]);
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int32_t cx = (k[0] + dx + g->nc[0]) % g->nc[0];
                int32_t cy = (k[1] + dy + g->nc[1]) % g->nc[1];
                int32_t cz = (k[2] + dz + g->nc[2]) % g->nc[2];
                int64_t c = cx + (int64_t)g->nc[0] * (cy + (int64_t)g->nc[1] * cz);
                for (int64_t s = g->start[c]; s < g->start[c + 1]; ++s) {
                    int64_t j = g->idx[s];
                    min_image(&x[3 * i], &x[3 * j], box, d);
                    cbuf_push(b, j, d, norm2(d));
                }
            }
}

static int cmp_cand(const void *pa, const void *pb)
{
    int64_t a = ((const cand_t *)pa)->j, b = ((const cand_t *)pb)->j;
    return (a > b) - (a < b);
}

/* ------------------------------------------------------------------------- */
/* Density and smoothing length (Eq. 6; readings R2-R5)                       */
/* ------------------------------------------------------------------------- */

/* rho(h) = sum_j m_j W(r_ij, h) and drho/dh over the neighbour set r^2 < 4h^2,
 * ascending j (R4); the count excludes j = i (R2). */
static void density_sums(const cbuf_t *all, cbuf_t *nb, const double *m, int64_t i,
                         double h, double *rho, double *drho_dh, int32_t *cnt)
{
    double R2 = 4.0 * h * h;
    nb->n = 0;
    for (int64_t s = 0; s < all->n; ++s)
        if (all->c[s].r2 < R2) cbuf_push(nb, all->c[s].j, all->c[s].d, all->c[s].r2);
    qsort(nb->c, (size_t)nb->n, sizeof(cand_t), cmp_cand);
    double sr = 0.0, sd = 0.0;
    int32_t k = 0;
    for (int64_t s = 0; s < nb->n; ++s) {
        double r = sqrt(nb->c[s].r2);
        sr += m[nb->c[s].j] * orc_W(r, h);
        sd += m[nb->c[s].j] * orc_dWdh(r, h);
        if (nb->c[s].j != i) ++k;
    }
    *rho = sr; *drho_dh = sd; *cnt = k;
}

void orc_density(int64_t n, const double *x, const double *m, const double *h_in,
                 const double *box, double eta, double h_cap, int newton_steps,
                 int brute, int64_t ntarget, const int64_t *targets,
                 double *rho, double *h_out, double *drho_dh, int32_t *nngb,
                 int32_t *flags, int64_t *pairs_all)
{
    grid_t g;
    int use_grid = !brute && grid_build(&g, n, x, box, 2.0 * h_cap);
    if (!use_grid) memset(&g, 0, sizeof(g));
    int64_t nt = targets ? ntarget : n;
    const double eta3 = eta * eta * eta;

#pragma omp parallel
    {
        cbuf_t all = {0}, nb = {0};
#pragma omp for schedule(dynamic, 64)
        for (int64_t t = 0; t < nt; ++t) {
            int64_t i = targets ? targets[t] : t;
            int32_t fl = 0;
            gather_candidates(&all, &g, !use_grid, n, x, box, i);
            double h = h_in[i];
            if (!isfinite(h) || !(h > 0.0)) { fl |= ORC_FLAG_NONFINITE; h = h_cap; }
            if (h > h_cap) { h = h_cap; fl |= ORC_FLAG_HCAP; }
            double r, dr;
            int32_t cnt;
            int64_t npairs = 0;     /* neighbour pairs summed over every pass */
            for (int s = 0; s < newton_steps; ++s) {
                density_sums(&all, &nb, m, i, h, &r, &dr, &cnt);
                npairs += cnt;
                /* R5: f(h) = rho(h) - m (eta/h)^3, f'(h) = drho/dh + 3 m eta^3 / h^4 */
                double f = r - m[i] * eta3 / (h * h * h);
                double fp = dr + 3.0 * m[i] * eta3 / (h * h * h * h);
                double hn = h;
                if (fp > 0.0 && isfinite(f) && isfinite(fp)) hn = h - f / fp;
                else fl |= ORC_FLAG_NEWTON;
                if (hn < 0.5 * h) hn = 0.5 * h;
                if (hn > 2.0 * h) hn = 2.0 * h;
                if (hn > h_cap) { hn = h_cap; fl |= ORC_FLAG_HCAP; }
                h = hn;
            }
            density_sums(&all, &nb, m, i, h, &r, &dr, &cnt);
            npairs += cnt;
            if (!isfinite(r)) fl |= ORC_FLAG_NONFINITE;
            rho[t] = r;
            if (h_out) h_out[t] = h;
            if (drho_dh) drho_dh[t] = dr;
            if (nngb) nngb[t] = cnt;
            if (flags) flags[t] = fl;
            if (pairs_all) pairs_all[t] = npairs;
        }
        free(all.c); free(nb.c);
    }
    if (use_grid) grid_free(&g);
}

/* ------------------------------------------------------------------------- */
/* Equation of state (R6)                                                     */
/* ------------------------------------------------------------------------- */

void orc_eos(int64_t n, const double *rho, const double *u, double gamma,
             double *P, double *c)
{
    for (int64_t i = 0; i < n; ++i) {
        P[i] = (gamma - 1.0) * rho[i] * u[i];
        c[i] = sqrt(gamma * P[i] / rho[i]);
    }
}

/* ------------------------------------------------------------------------- */
/* Symmetric hydro force with artificial viscosity (Eq. 7, Eq. 5; R7-R9)      */
/* ------------------------------------------------------------------------- */

/* one interacting pair (r2 > 0) of the force sums: adds particle j's terms to
 * the acceleration acc[0..2] and du/dt of particle i; d = x_i - x_j */
static void force_pair(int64_t i, int64_t j, const double *d, double r2, const double *v,
                       const double *m, const double *h, const double *rho, const double *P,
                       const double *c, double alpha, double beta, double eps, double *acc,
                       double *du)
{
    const double Pi_rho2 = P[i] / (rho[i] * rho[i]);
    double r = sqrt(r2);
    double hb = 0.5 * (h[i] + h[j]);
    double gw = orc_dWdr(r, hb) / r;  /* grad_i W = d * gw */
    double vij[3] = { v[3 * i] - v[3 * j], v[3 * i + 1] - v[3 * j + 1],
                      v[3 * i + 2] - v[3 * j + 2] };
    double vdotr = vij[0] * d[0] + vij[1] * d[1] + vij[2] * d[2];
    /* R8: Monaghan viscosity, only for approaching pairs */
    double visc = 0.0;
    if (vdotr < 0.0) {
        double mu = hb * vdotr / (r2 + eps * hb * hb);
        double cbar = 0.5 * (c[i] + c[j]);
        double rhobar = 0.5 * (rho[i] + rho[j]);
        visc = (-alpha * cbar * mu + beta * mu * mu) / rhobar;
    }
    double Pj_rho2 = P[j] / (rho[j] * rho[j]);
    double fac = m[j] * (Pi_rho2 + Pj_rho2 + visc) * gw;
    acc[0] -= fac * d[0];
    acc[1] -= fac * d[1];
    acc[2] -= fac * d[2];
    /* Eq. 5: du/dt = (P_i/rho_i^2) sum_j m_j v_ij . grad W + 1/2 sum_j m_j Pi_ij v_ij . grad W */
    *du += m[j] * (Pi_rho2 + 0.5 * visc) * (vdotr * gw);
}

void orc_force(int64_t n, const double *x, const double *v, const double *m,
               const double *h, const double *rho, const double *P, const double *c,
               const double *box, double alpha, double beta, double eps,
               int brute, int64_t ntarget, const int64_t *targets,
               double *a, double *dudt, int32_t *nngb)
{
    double hmax = 0.0;
    for (int64_t i = 0; i < n; ++i) if (h[i] > hmax) hmax = h[i];
    grid_t g;
    int use_grid = !brute && grid_build(&g, n, x, box, 2.0 * hmax);
    if (!use_grid) memset(&g, 0, sizeof(g));
    int64_t nt = targets ? ntarget : n;

#pragma omp parallel
    {
        cbuf_t all = {0}, nb = {0};
#pragma omp for schedule(dynamic, 64)
        for (int64_t t = 0; t < nt; ++t) {
            int64_t i = targets ? targets[t] : t;
            gather_candidates(&all, &g, !use_grid, n, x, box, i);
            nb.n = 0;
            for (int64_t s = 0; s < all.n; ++s) {
                int64_t j = all.c[s].j;
                double hs = h[i] + h[j];          /* r < 2 h_ij = h_i + h_j (R7) */
                if (j != i && all.c[s].r2 < hs * hs) cbuf_push(&nb, j, all.c[s].d, all.c[s].r2);
            }
            qsort(nb.c, (size_t)nb.n, sizeof(cand_t), cmp_cand);
            double acc[3] = {0.0, 0.0, 0.0}, du = 0.0;
            for (int64_t s = 0; s < nb.n; ++s) {
                double r2 = nb.c[s].r2;
                if (r2 == 0.0) continue;        /* coincident pair: grad W = 0 */
                force_pair(i, nb.c[s].j, nb.c[s].d, r2, v, m, h, rho, P, c, alpha, beta, eps, acc, &du);
            }
            a[3 * t + 0] = acc[0]; a[3 * t + 1] = acc[1]; a[3 * t + 2] = acc[2];
            dudt[t] = du;
            if (nngb) nngb[t] = (int32_t)nb.n;
        }
        free(all.c); free(nb.c);
    }
    if (use_grid) grid_free(&g);
}

/* ------------------------------------------------------------------------- */
/* Buffers of co-located particles (Section 6, the benchmark's grouping)      */
/* ------------------------------------------------------------------------- */
/* The paper's benchmark keeps particles in contiguous buffers of B spatially
 * co-located particles and evaluates the quadratic kernels over every pair of
 * a buffer (64 x 64 for B = 64).  Buffer b holds particles [bB, min((b+1)B, n));
 * separations are minimum images; partners in ascending j.
 * Density: Eq. 6 restricted to the buffer, self included, h fixed, then the
 * EOS (R6).  Force: Eq. 7 and Eq. 5 restricted to the buffer, pairs
 * r < h_i + h_j (R7-R9).  nngb counts partners j != i within the support. */

void orc_buffer_density(int64_t n, int32_t B, const double *x, const double *m,
                        const double *h, const double *u, const double *box, double gamma,
                        double *rho, double *P, double *c, int32_t *nngb)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const int64_t j0 = (i / B) * B;
        const int64_t j1 = j0 + B < n ? j0 + B : n;
        double sr = 0.0;
        int32_t k = 0;
        for (int64_t j = j0; j < j1; ++j) {
            double d[3];
            min_image(x + 3 * i, x + 3 * j, box, d);
            double r2 = norm2(d);
            if (!(r2 < 4.0 * h[i] * h[i])) continue;
            sr += m[j] * orc_W(sqrt(r2), h[i]);
            if (j != i) ++k;
        }
        rho[i] = sr;
        P[i] = (gamma - 1.0) * sr * u[i];
        c[i] = sqrt(gamma * P[i] / sr);
        if (nngb) nngb[i] = k;
    }
}

void orc_buffer_force(int64_t n, int32_t B, const double *x, const double *v, const double *m,
                      const double *h, const double *rho, const double *P, const double *c,
                      const double *box, double alpha, double beta, double eps,
                      double *a, double *dudt, int32_t *nngb)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const int64_t j0 = (i / B) * B;
        const int64_t j1 = j0 + B < n ? j0 + B : n;
        double acc[3] = {0.0, 0.0, 0.0}, du = 0.0;
        int32_t k = 0;
        for (int64_t j = j0; j < j1; ++j) {
            if (j == i) continue;
            double d[3];
            min_image(x + 3 * i, x + 3 * j, box, d);
            double r2 = norm2(d);
            double hs = h[i] + h[j];
            if (!(r2 < hs * hs)) continue;
            ++k;
            if (r2 == 0.0) continue;            /* coincident pair: grad W = 0 */
            force_pair(i, j, d, r2, v, m, h, rho, P, c, alpha, beta, eps, acc, &du);
        }
        a[3 * i + 0] = acc[0]; a[3 * i + 1] = acc[1]; a[3 * i + 2] = acc[2];
        dudt[i] = du;
        if (nngb) nngb[i] = k;
    }
}

/* ------------------------------------------------------------------------- */
/* Kick / drift (R10)                                                         */
/* ------------------------------------------------------------------------- */

void orc_kick_drift(int64_t n, double *x, double *v, const double *a, double *u,
                    const double *dudt, double dt_kick, double dt_drift,
                    const double *box)
{
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) v[3 * i + k] += a[3 * i + k] * dt_kick;
        u[i] += dudt[i] * dt_kick;
        for (int k = 0; k < 3; ++k) {
            double y = x[3 * i + k] + v[3 * i + k] * dt_drift;
            y -= box[k] * floor(y / box[k]);
            if (y >= box[k]) y = 0.0;            /* rounding at the upper edge */
            x[3 * i + k] = y;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Ball query helper (for sampled checks on large inputs)                     */
/* ------------------------------------------------------------------------- */

int64_t orc_ball_mark(int64_t n, const double *x, const double *box, double radius,
                      int64_t ntarget, const int64_t *targets, uint8_t *mark)
{
    grid_t g;
    int use_grid = grid_build(&g, n, x, box, radius);
    if (!use_grid) memset(&g, 0, sizeof(g));
    memset(mark, 0, (size_t)n);
    cbuf_t all = {0};
    double R2 = radius * radius;
    for (int64_t t = 0; t < ntarget; ++t) {
        gather_candidates(&all, &g, !use_grid, n, x, box, targets[t]);
        for (int64_t s = 0; s < all.n; ++s)
            if (all.c[s].r2 < R2) mark[all.c[s].j] = 1;
        mark[targets[t]] = 1;
    }
    free(all.c);
    if (use_grid) grid_free(&g);
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) k += mark[i];
    return k;
}

/* ------------------------------------------------------------------------- */
/* Quantisers (Table 2; R11)                                                  */
/* ------------------------------------------------------------------------- */

uint32_t orc_f32_bits(double d)
{
    float f = (float)d;                 /* IEEE 754 conversion: round to nearest even */
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
}

double orc_f32_value(uint32_t bits)
{
    float f;
    memcpy(&f, &bits, 4);
    return (double)f;
}

/* binary32 -> binary16, round to nearest, ties to even, IEEE subnormals,
 * overflow to infinity, NaN kept quiet. */
uint16_t orc_f16_from_f32(uint32_t fb)
{
    uint32_t sign = (fb >> 16) & 0x8000u;
    uint32_t e = (fb >> 23) & 0xFFu;
    uint32_t man = fb & 0x7FFFFFu;
    if (e == 0xFFu) return (uint16_t)(sign | 0x7C00u | (man ? (0x200u | (man >> 13)) : 0u));
    if (e == 0u) return (uint16_t)sign;     /* |x| < 2^-126: far below half precision */
    int32_t E = (int32_t)e - 127;           /* unbiased exponent */
    uint32_t m24 = man | 0x800000u;         /* value = m24 * 2^(E-23) */
    uint32_t shift, kept;
    if (E >= -14) {                         /* normal half, or overflow */
        if (E > 15) return (uint16_t)(sign | 0x7C00u);
        shift = 13;
        kept = ((uint32_t)(E + 15) << 10) | ((m24 >> 13) & 0x3FFu);
    } else {                                /* subnormal half: units of 2^-24 */
        shift = (uint32_t)(-E - 1);
        if (shift > 24) return (uint16_t)sign;  /* below half the smallest subnormal */
        kept = m24 >> shift;
    }
    uint32_t rem = m24 & ((1u << shift) - 1u);
    uint32_t halfway = 1u << (shift - 1);
    /* adding 1 carries from the mantissa into the exponent field when needed */
    if (rem > halfway || (rem == halfway && (kept & 1u))) kept += 1u;
    if (kept >= 0x7C00u) return (uint16_t)(sign | 0x7C00u);
    return (uint16_t)(sign | kept);
}

uint32_t orc_f32_from_f16(uint16_t hb)
{
    uint32_t sign = ((uint32_t)hb & 0x8000u) << 16;
    uint32_t e = ((uint32_t)hb >> 10) & 0x1Fu;
    uint32_t man = (uint32_t)hb & 0x3FFu;
    if (e == 0x1F) return sign | 0x7F800000u | (man << 13);
    if (e == 0) {
        if (man == 0) return sign;
        /* subnormal: value = man * 2^-24; normalise */
        int32_t k = 0;
        while (!(man & 0x400u)) { man <<= 1; ++k; }
        man &= 0x3FFu;
        return sign | ((uint32_t)(127 - 15 + 1 - k) << 23) | (man << 13);
    }
    return sign | ((e - 15 + 127) << 23) | (man << 13);
}

/* binary32 -> bfloat16 (top 16 bits), round to nearest even, NaN kept quiet */
uint16_t orc_bf16_from_f32(uint32_t fb)
{
    if ((fb & 0x7F800000u) == 0x7F800000u && (fb & 0x7FFFFFu))
        return (uint16_t)((fb >> 16) | 0x40u);
    uint32_t lower = fb & 0xFFFFu;
    uint32_t upper = fb >> 16;
    if (lower > 0x8000u || (lower == 0x8000u && (upper & 1u))) upper += 1u;
    return (uint16_t)upper;
}

uint32_t orc_f32_from_bf16(uint16_t bb)
{
    return (uint32_t)bb << 16;
}

/* Table 2, "31..17" column: sign, 8 exponent bits and the top `mant_bits`
 * mantissa bits of the binary32 value, the rest dropped (truncation toward
 * zero).  A NaN keeps its quiet bit so that it stays a NaN. */
uint32_t orc_trunc_code(uint32_t fb, int mant_bits)
{
    int drop = 23 - mant_bits;
    if ((fb & 0x7F800000u) == 0x7F800000u && (fb & 0x7FFFFFu)) fb |= 0x400000u;
    return fb >> drop;
}

uint32_t orc_f32_from_trunc(uint32_t code, int mant_bits)
{
    return code << (23 - mant_bits);
}

int orc_fmt_bits(int fmt)
{
    if (fmt > 100 && fmt <= 122) return 9 + (fmt - 100);
    switch (fmt) {
    case ORC_FMT_FP32: return 32;
    case ORC_FMT_BF16: return 16;
    case ORC_FMT_FP16: return 16;
    case ORC_FMT_M16:  return 1 + 8 + 16;
    case ORC_FMT_M10:  return 1 + 8 + 10;
    default: return 0;
    }
}

void orc_quantize(int64_t n, const double *in, int fmt, double *value, uint32_t *code)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t fb = orc_f32_bits(in[i]);
        uint32_t cd, back;
        switch (fmt) {
        case ORC_FMT_BF16: cd = orc_bf16_from_f32(fb); back = orc_f32_from_bf16((uint16_t)cd); break;
        case ORC_FMT_FP16: cd = orc_f16_from_f32(fb); back = orc_f32_from_f16((uint16_t)cd); break;
        case ORC_FMT_M16:  cd = orc_trunc_code(fb, 16); back = orc_f32_from_trunc(cd, 16); break;
        case ORC_FMT_M10:  cd = orc_trunc_code(fb, 10); back = orc_f32_from_trunc(cd, 10); break;
        default:
            if (fmt > 100 && fmt <= 122) {        /* ORC_FMT_TRUNC(n) */
                cd = orc_trunc_code(fb, fmt - 100);
                back = orc_f32_from_trunc(cd, fmt - 100);
            } else {
                cd = fb;
                back = fb;
            }
            break;
        }
        if (value) value[i] = orc_f32_value(back);
        if (code) code[i] = cd;
    }
}

/* Table 2, total widths 63..33: the double layout (sign, 11 exponent bits)
 * with its mantissa truncated toward zero to `mant` bits (0..52; 52 keeps
 * every value).  Infinities and NaNs pass unchanged. */
void orc_trunc64(int64_t n, const double *in, int mant, double *out)
{
    const uint64_t keep = mant >= 52 ? ~0ull : ~((1ull << (52 - mant)) - 1ull);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t b;
        memcpy(&b, &in[i], 8);
        if (((b >> 52) & 0x7FFull) != 0x7FFull) b &= keep;
        memcpy(&out[i], &b, 8);
    }
}

/* Table 2, total widths 15 and below: the half layout (sign, 5 exponent
 * bits) with its mantissa truncated toward zero to `mant` bits (0..10): the
 * value is first rounded to half (through single, as ORC_FMT_FP16), then the
 * low 10 - mant mantissa bits of the half are cleared.  Infinities and NaNs
 * keep their class. */
void orc_trunc_half(int64_t n, const double *in, int mant, double *out)
{
    const uint16_t keep = (uint16_t)(mant >= 10 ? 0xFFFFu : ~((1u << (10 - mant)) - 1u));
    for (int64_t i = 0; i < n; ++i) {
        uint16_t h = orc_f16_from_f32(orc_f32_bits(in[i]));
        if ((h & 0x7C00u) != 0x7C00u) h &= keep;
        out[i] = orc_f32_value(orc_f32_from_f16(h));
    }
}

/* Sec. 3.2: value k occupies bits [k*B, (k+1)*B) of a little-endian stream of
 * 32-bit words.  `words` must hold ceil(n*B/32) entries and is overwritten. */
void orc_pack_bits(int64_t n, const uint32_t *codes, int bits, uint32_t *words)
{
    int64_t nw = (n * bits + 31) / 32;
    for (int64_t w = 0; w < nw; ++w) words[w] = 0u;
    for (int64_t k = 0; k < n; ++k) {
        for (int b = 0; b < bits; ++b) {
            if ((codes[k] >> b) & 1u) {
                int64_t pos = k * bits + b;
                words[pos / 32] |= 1u << (pos % 32);
            }
        }
    }
}

void orc_unpack_bits(int64_t n, const uint32_t *words, int bits, uint32_t *codes)
{
    for (int64_t k = 0; k < n; ++k) {
        uint32_t c = 0;
        for (int b = 0; b < bits; ++b) {
            int64_t pos = k * bits + b;
            if ((words[pos / 32] >> (pos % 32)) & 1u) c |= 1u << b;
        }
        codes[k] = c;
    }
}
