/*
 * oracle.c -- plain FP64 CPU reference for the relativistic line-of-sight sum.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the GPU library is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code, header, table or helper with
 * the CUDA path (no DDA, no bricks, no FP32 arithmetic), and the CUDA path must
 * never call it.
 *
 * What it computes (Whitehead, Elley & Everett, "cuDART"):
 *
 *   I_nu = (nu/nu'_0)^alpha * sum_m sum_n W_{n,m} D_{n,m}^{2-alpha} j'_{n,m} ds_n
 *                                                        (Eq. 19, Sec. 2.5)
 *
 * written out as its plain definition:
 *   1. an orthographic ray through each pixel centre (camera readings A4, A5,
 *      A12 below);
 *   2. the ray is clipped to the grid box (the cuboid-ray test of Sec. 2.4);
 *   3. EVERY face-plane crossing x_i = origin_i + k dx_i inside the box is
 *      enumerated for each axis, all crossings are sorted and merged, and
 *      zero-length gaps are dropped -- this is the set of cells n crossed by the
 *      ray and their line elements ds_n (Sec. 2.3, Eq. 4; Sec. 2.4) without any
 *      traversal algorithm;
 *   4. each segment's cell is the floor of its midpoint position;
 *   5. the local evaluation time is t_bar = t_obs - s/c (Eq. 2), taken at the
 *      chord midpoint, with s measured from the image plane through the view
 *      centre (readings A3, A4);
 *   6. the temporal weights are the linear kernel W_{n,m} = 1 - delta_{n,m} for
 *      m in {m_bar, m_bar+1}, zero otherwise (Eqs. 6-8, Sec. 2.3), summed over
 *      the stored snapshots m = 0 .. M-1 only (Eq. 9; reading A6); without
 *      lookback every cell is read at t_obs (Eq. 3, Eq. 10) with the epoch
 *      coordinate clamped to the stored range (reading A8);
 *   7. D = 1/(Gamma (1 + beta . s_hat)), Gamma = 1/sqrt(1 - beta^2) (Eq. 14),
 *      raised to 2 - alpha (Eqs. 18-19); D = 1 with beaming off (routine A of
 *      Sec. 3);
 *   8. the sum is scaled by (nu/nu'_0)^alpha (Eqs. 19-20).
 *
 * Readings where the paper is silent (numbered as in the design notes):
 *   A3  t_bar of a cell is evaluated at its chord midpoint.  Optional variant
 *       `split_at_nodes` cuts a chord where its epoch coordinate passes an
 *       integer, so that the piecewise-linear weight is integrated exactly.
 *   A4  s is measured from the plane through the view centre, normal to s_hat.
 *   A5  orthographic projection (observer at infinity).
 *   A6  the sum over m in Eq. 9 runs over the stored snapshots.  A time
 *       within one cadence before t_0 (after t_{M-1}) keeps the weight
 *       1 - delta of the first (last) snapshot, fading linearly to zero; a time
 *       further out contributes nothing.  The sum is continuous in t_bar.
 *   A8  fast light: every cell at t_obs, epoch coordinate clamped to [0, M-1].
 *   A11 a point exactly on a face belongs to the cell on the + side (floor).
 *   A12 pixel (p, q) centre at ((p + 1/2 - W/2) h_u, (q + 1/2 - H/2) h_v) on the
 *       image axes (e_u, e_v); e_v is `up` projected normal to s_hat; e_u =
 *       s_hat x e_v; row q = 0 is the bottom row; image[q][p].
 *
 * Layouts: j is [M][nz][ny][nx], beta is [M][nz][ny][nx][3], x fastest,
 * either float64 or float32 (promoted to double on read).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_INVALID 1
#define ORC_ERR_NOMEM 2

enum { ORC_F64 = 0, ORC_F32 = 1 };

typedef struct {
    int32_t n[3];       /* cells along x, y, z                          */
    double origin[3];   /* lower corner of cell (0, 0, 0)               */
    double dx[3];       /* cell edge along each axis (need not be equal) */
    int32_t n_epochs;   /* M snapshots                                   */
    double t0, dt;      /* epoch m is at t_m = t0 + m dt (Eq. 5)         */
} orc_grid;

typedef struct {
    const void *j;      /* rest-frame emissivity j'  [M][nz][ny][nx]     */
    const void *beta;   /* velocity / c              [M][nz][ny][nx][3]  */
    int32_t dtype;      /* ORC_F64 or ORC_F32                            */
} orc_fields;

typedef struct {
    double dir[3];      /* s_hat: viewing direction, into the scene      */
    double up[3];       /* image "up" before projection                  */
    double center[3];   /* image-plane centre, s = 0 there               */
    double t_obs;       /* observer time                                 */
    double c;           /* signal speed (cells per unit time); may be inf*/
    double alpha;       /* rest-frame spectral slope, j' ~ nu'^alpha     */
    double nu_ratio;    /* nu / nu'_0                                    */
    int32_t beaming;    /* apply D^(2 - alpha)                           */
    int32_t lookback;   /* evaluate fields at t_bar = t_obs - s/c        */
    int32_t width, height;
    double fov_u, fov_v;/* image extent along e_u, e_v (world units)     */
    int32_t split_at_nodes; /* reading A3 variant, see header            */
} orc_view;

static double load(const void *p, int32_t dtype, size_t i)
{
    return dtype == ORC_F64 ? ((const double *)p)[i] : (double)((const float *)p)[i];
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Orthonormal camera basis (reading A12). */
static int camera_basis(const orc_view *v, double sh[3], double eu[3], double ev[3])
{
    double nd = sqrt(v->dir[0] * v->dir[0] + v->dir[1] * v->dir[1] + v->dir[2] * v->dir[2]);
    if (!(nd > 0.0) || !isfinite(nd)) return ORC_ERR_INVALID;
    for (int i = 0; i < 3; ++i) sh[i] = v->dir[i] / nd;
    double us = v->up[0] * sh[0] + v->up[1] * sh[1] + v->up[2] * sh[2];
    for (int i = 0; i < 3; ++i) ev[i] = v->up[i] - us * sh[i];
    double nv = sqrt(ev[0] * ev[0] + ev[1] * ev[1] + ev[2] * ev[2]);
    if (!(nv > 1e-12)) return ORC_ERR_INVALID;
    for (int i = 0; i < 3; ++i) ev[i] /= nv;
    eu[0] = sh[1] * ev[2] - sh[2] * ev[1];
    eu[1] = sh[2] * ev[0] - sh[0] * ev[2];
    eu[2] = sh[0] * ev[1] - sh[1] * ev[0];
    return ORC_OK;
}

/* W_{n,m} D_{n,m}^{2-alpha} j'_{n,m}, summed over the stored m, for one cell
 * at epoch coordinate u = (t_bar - t0)/dt (Eqs. 6-9 and 14, 19).  *inside is
 * set when at least one stored snapshot has a nonzero weight. */
static double cell_value(const orc_grid *g, const orc_fields *f, const orc_view *v,
                         const double sh[3], size_t cell, double u, int *inside)
{
    const int M = g->n_epochs;
    const size_t ncell = (size_t)g->n[0] * g->n[1] * g->n[2];
    if (v->lookback) {
        if (!(u > -1.0 && u < (double)M)) { *inside = 0; return 0.0; }
    } else {
        if (u < 0.0) u = 0.0;
        if (u > (double)(M - 1)) u = (double)(M - 1);
    }
    *inside = 1;
    double mbar = floor(u);
    double sum = 0.0;
    for (int k = 0; k < 2; ++k) {
        double m = mbar + k;
        if (m < 0.0 || m > (double)(M - 1)) continue;   /* stored snapshots only */
        double w = 1.0 - fabs(u - m);          /* Eq. 7 with Eq. 6 */
        if (!(w > 0.0)) continue;
        size_t idx = (size_t)m * ncell + cell;
        double jp = load(f->j, f->dtype, idx);
        double boosted = jp;
        if (v->beaming) {
            double bx = load(f->beta, f->dtype, 3 * idx + 0);
            double by = load(f->beta, f->dtype, 3 * idx + 1);
            double bz = load(f->beta, f->dtype, 3 * idx + 2);
            double b2 = bx * bx + by * by + bz * bz;
            double gamma = 1.0 / sqrt(1.0 - b2);                     /* Eq. 14 */
            double D = 1.0 / (gamma * (1.0 + bx * sh[0] + by * sh[1] + bz * sh[2]));
            boosted = pow(D, 2.0 - v->alpha) * jp;                   /* Eq. 19 */
        }
        sum += w * boosted;
    }
    return sum;
}

/* Epoch coordinate of a point at distance s along the ray (Eq. 2, Eq. 5). */
static double epoch_coord(const orc_grid *g, const orc_view *v, double s)
{
    double tbar = v->lookback ? v->t_obs - s / v->c : v->t_obs;
    return (tbar - g->t0) / g->dt;
}

/* One pixel: returns the intensity and the number of positive-length cell
 * chords with a nonzero temporal weight (the "cell-samples"). */
static double render_pixel(const orc_grid *g, const orc_fields *f, const orc_view *v,
                           const double sh[3], const double eu[3], const double ev[3],
                           int p, int q, double *crossings, int64_t *count)
{
    double hu = v->fov_u / v->width, hv = v->fov_v / v->height;
    double a = (p + 0.5 - 0.5 * v->width) * hu;
    double b = (q + 0.5 - 0.5 * v->height) * hv;
    double r0[3];
    for (int i = 0; i < 3; ++i) r0[i] = v->center[i] + a * eu[i] + b * ev[i];

    /* Clip to the box [origin, origin + n dx) (Sec. 2.4 entry test). */
    double s_in = -INFINITY, s_out = INFINITY;
    for (int i = 0; i < 3; ++i) {
        double lo = g->origin[i], hi = g->origin[i] + g->n[i] * g->dx[i];
        if (sh[i] == 0.0) {
            if (r0[i] < lo || r0[i] >= hi) { *count = 0; return 0.0; }
        } else {
            double t1 = (lo - r0[i]) / sh[i], t2 = (hi - r0[i]) / sh[i];
            double tmin = t1 < t2 ? t1 : t2, tmax = t1 < t2 ? t2 : t1;
            if (tmin > s_in) s_in = tmin;
            if (tmax < s_out) s_out = tmax;
        }
    }
    if (!(s_out > s_in)) { *count = 0; return 0.0; }

    /* Every interior face-plane crossing, all axes. */
    int nc = 0;
    crossings[nc++] = s_in;
    for (int i = 0; i < 3; ++i) {
        if (sh[i] == 0.0) continue;
        for (int k = 1; k < g->n[i]; ++k) {
            double s = (g->origin[i] + k * g->dx[i] - r0[i]) / sh[i];
            if (s > s_in && s < s_out) crossings[nc++] = s;
        }
    }
    crossings[nc++] = s_out;
    qsort(crossings, (size_t)nc, sizeof(double), cmp_double);

    double acc = 0.0;
    int64_t samples = 0;
    for (int c = 0; c + 1 < nc; ++c) {
        double s0 = crossings[c], s1 = crossings[c + 1];
        if (!(s1 > s0)) continue;                 /* merged duplicate plane */
        double mid = 0.5 * (s0 + s1);
        size_t cell = 0, stride = 1;
        for (int i = 0; i < 3; ++i) {
            double xi = r0[i] + mid * sh[i];
            long k = (long)floor((xi - g->origin[i]) / g->dx[i]);
            if (k < 0) k = 0;
            if (k > g->n[i] - 1) k = g->n[i] - 1;
            cell += (size_t)k * stride;
            stride *= (size_t)g->n[i];
        }
        int inside = 0;
        double contrib = 0.0;
        if (v->split_at_nodes && v->lookback && isfinite(v->c)) {
            /* Cut the chord where the epoch coordinate passes an integer, so
             * that the piecewise-linear weight is integrated exactly. */
            double u0 = epoch_coord(g, v, s0), u1 = epoch_coord(g, v, s1);
            double ulo = u0 < u1 ? u0 : u1, uhi = u0 < u1 ? u1 : u0;
            double cuts[64];
            int ncut = 0;
            cuts[ncut++] = s0;
            for (double k = floor(ulo) + 1.0; k < uhi && ncut < 62; k += 1.0) {
                double sk = v->c * (v->t_obs - g->t0 - k * g->dt);
                if (sk > s0 && sk < s1) cuts[ncut++] = sk;
            }
            cuts[ncut++] = s1;
            qsort(cuts, (size_t)ncut, sizeof(double), cmp_double);
            for (int t = 0; t + 1 < ncut; ++t) {
                double m2 = 0.5 * (cuts[t] + cuts[t + 1]);
                int in2 = 0;
                double val = cell_value(g, f, v, sh, cell, epoch_coord(g, v, m2), &in2);
                contrib += val * (cuts[t + 1] - cuts[t]);
                inside |= in2;
            }
        } else {
            double val = cell_value(g, f, v, sh, cell, epoch_coord(g, v, mid), &inside);
            contrib = val * (s1 - s0);
        }
        acc += contrib;
        samples += inside;
    }
    *count = samples;
    return pow(v->nu_ratio, v->alpha) * acc;   /* Eq. 19 prefactor, Eq. 20 */
}

static int validate(const orc_grid *g, const orc_fields *f, const orc_view *v)
{
    if (!g || !f || !v || !f->j || (v->beaming && !f->beta)) return ORC_ERR_INVALID;
    for (int i = 0; i < 3; ++i)
        if (g->n[i] < 1 || !(g->dx[i] > 0.0)) return ORC_ERR_INVALID;
    if (g->n_epochs < 1 || !(g->dt > 0.0)) return ORC_ERR_INVALID;
    if (v->width < 1 || v->height < 1 || !(v->fov_u > 0.0) || !(v->fov_v > 0.0)) return ORC_ERR_INVALID;
    if (v->lookback && !(v->c > 0.0)) return ORC_ERR_INVALID;
    if (f->dtype != ORC_F64 && f->dtype != ORC_F32) return ORC_ERR_INVALID;
    return ORC_OK;
}

/* Render a full image[height][width]; counts (optional) receives the number
 * of cell-samples per pixel.  n_threads <= 0 uses every available thread. */
int orc_render(const orc_grid *g, const orc_fields *f, const orc_view *v,
               double *image, int64_t *counts, int32_t n_threads)
{
    int rc = validate(g, f, v);
    if (rc) return rc;
    double sh[3], eu[3], ev[3];
    if ((rc = camera_basis(v, sh, eu, ev))) return rc;
    const int maxc = g->n[0] + g->n[1] + g->n[2] + 4;
    int failed = 0;
#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel num_threads(nt)
#endif
    {
        double *cr = (double *)malloc(sizeof(double) * (size_t)maxc);
        if (!cr) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            failed = 1;
        }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int q = 0; q < v->height; ++q) {
            if (!cr) continue;
            for (int p = 0; p < v->width; ++p) {
                int64_t cnt = 0;
                double val = render_pixel(g, f, v, sh, eu, ev, p, q, cr, &cnt);
                image[(size_t)q * v->width + p] = val;
                if (counts) counts[(size_t)q * v->width + p] = cnt;
            }
        }
        free(cr);
    }
    (void)n_threads;
    return failed ? ORC_ERR_NOMEM : ORC_OK;
}

/* Render a list of pixels given as (p, q) pairs; used for sampled checks of
 * full-size images. */
int orc_render_pixels(const orc_grid *g, const orc_fields *f, const orc_view *v,
                      const int32_t *pq, int64_t n_pix, double *out, int64_t *counts,
                      int32_t n_threads)
{
    int rc = validate(g, f, v);
    if (rc) return rc;
    double sh[3], eu[3], ev[3];
    if ((rc = camera_basis(v, sh, eu, ev))) return rc;
    const int maxc = g->n[0] + g->n[1] + g->n[2] + 4;
    int failed = 0;
#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel num_threads(nt)
#endif
    {
        double *cr = (double *)malloc(sizeof(double) * (size_t)maxc);
        if (!cr) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            failed = 1;
        }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t k = 0; k < n_pix; ++k) {
            if (!cr) continue;
            int p = pq[2 * k], q = pq[2 * k + 1];
            int64_t cnt = 0;
            double val = 0.0;
            if (p >= 0 && p < v->width && q >= 0 && q < v->height)
                val = render_pixel(g, f, v, sh, eu, ev, p, q, cr, &cnt);
            out[k] = val;
            if (counts) counts[k] = cnt;
        }
        free(cr);
    }
    (void)n_threads;
    return failed ? ORC_ERR_NOMEM : ORC_OK;
}

/* Threads the oracle would use by default. */
int32_t orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
