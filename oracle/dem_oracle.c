/*
 * dem_oracle.c -- plain FP64 CPU oracle of the per-timestep DEM contact pipeline of
 * arXiv 2311.04648 (Chrono DEM-Engine).  TEST INFRASTRUCTURE ONLY; see dem_oracle.h.
 *
 * Deliberately slow and literal: brute-force O(N^2) contact search every step, one
 * contact at a time in lexicographic (i, j) order, no blocking or fusion.  Build with
 * -O2 -ffp-contract=off.
 */
#include "dem_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ small vectors */

static double dot3(const double a[3], const double b[3]) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }

static void cross3(const double a[3], const double b[3], double out[3])
{
    double c0 = a[1] * b[2] - a[2] * b[1];
    double c1 = a[2] * b[0] - a[0] * b[2];
    double c2 = a[0] * b[1] - a[1] * b[0];
    out[0] = c0; out[1] = c1; out[2] = c2;
}

static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }

/* Rotation matrix of a unit quaternion (w, x, y, z), row-major. */
static void quat_matrix(const double q[4], double R[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double xx = x * x, yy = y * y, zz = z * z;
    double xy = x * y, xz = x * z, yz = y * z;
    double wx = w * x, wy = w * y, wz = w * z;
    R[0] = 1.0 - 2.0 * (yy + zz); R[1] = 2.0 * (xy - wz);       R[2] = 2.0 * (xz + wy);
    R[3] = 2.0 * (xy + wz);       R[4] = 1.0 - 2.0 * (xx + zz); R[5] = 2.0 * (yz - wx);
    R[6] = 2.0 * (xz - wy);       R[7] = 2.0 * (yz + wx);       R[8] = 1.0 - 2.0 * (xx + yy);
}

static void mat_vec(const double R[9], const double a[3], double out[3])
{
    double o0 = (R[0] * a[0] + R[1] * a[1]) + R[2] * a[2];
    double o1 = (R[3] * a[0] + R[4] * a[1]) + R[5] * a[2];
    double o2 = (R[6] * a[0] + R[7] * a[1]) + R[8] * a[2];
    out[0] = o0; out[1] = o1; out[2] = o2;
}

static void mat_tvec(const double R[9], const double a[3], double out[3])
{
    double o0 = (R[0] * a[0] + R[3] * a[1]) + R[6] * a[2];
    double o1 = (R[1] * a[0] + R[4] * a[1]) + R[7] * a[2];
    double o2 = (R[2] * a[0] + R[5] * a[1]) + R[8] * a[2];
    out[0] = o0; out[1] = o1; out[2] = o2;
}

/* Hamilton product a (x) b. */
static void quat_mul(const double a[4], const double b[4], double out[4])
{
    double w = ((a[0] * b[0] - a[1] * b[1]) - a[2] * b[2]) - a[3] * b[3];
    double x = ((a[0] * b[1] + a[1] * b[0]) + a[2] * b[3]) - a[3] * b[2];
    double y = ((a[0] * b[2] - a[1] * b[3]) + a[2] * b[0]) + a[3] * b[1];
    double z = ((a[0] * b[3] + a[1] * b[2]) - a[2] * b[1]) + a[3] * b[0];
    out[0] = w; out[1] = x; out[2] = y; out[3] = z;
}

/* ------------------------------------------------------------------ materials */

/* E* and G* of a contact.  The paper calls a routine for this (Sec. 4.2.1, material
 * properties) without printing it; the reading adopted is the standard Hertz-Mindlin
 * combination 1/E* = sum (1 - nu^2)/E and 1/G* = sum 2 (2 - nu)(1 + nu)/E. */
void orc_effective_moduli(double E_a, double nu_a, double E_b, double nu_b, double *E_star, double *G_star)
{
    double ia = (1.0 - nu_a * nu_a) / E_a;
    double ib = (1.0 - nu_b * nu_b) / E_b;
    *E_star = 1.0 / (ia + ib);
    double ga = 2.0 * (2.0 - nu_a) * (1.0 + nu_a) / E_a;
    double gb = 2.0 * (2.0 - nu_b) * (1.0 + nu_b) / E_b;
    *G_star = 1.0 / (ga + gb);
}

/* Damping ratio from the restitution coefficient, CoR clamped below at 1e-12
 * (Sec. 4.2.1, normal force): beta = ln e / sqrt(ln^2 e + pi^2) <= 0. */
static double damping_beta(double cor)
{
    double e = cor < 1e-12 ? 1e-12 : cor;
    double le = log(e);
    return le / sqrt(le * le + ORC_PI * ORC_PI);
}

/* ------------------------------------------------------------------ history */

typedef struct {
    int64_t n, cap;
    int64_t *i, *j;      /* j >= 0 sphere, j < 0 wall -1-j */
    double *ut;          /* 3 per entry */
    double *age;         /* time in contact, 1 per entry */
    double *wc;          /* further model wildcards, 4 per entry */
} orc_hist;

/* Sort key of the partner: spheres first by id, then walls by wall id. */
static int64_t partner_key(int64_t j) { return j >= 0 ? j : ((int64_t)1 << 62) + (-1 - j); }

static int key_less(int64_t ia, int64_t ja, int64_t ib, int64_t jb)
{
    if (ia != ib) return ia < ib;
    return partner_key(ja) < partner_key(jb);
}

void *orc_history_new(void)
{
    orc_hist *h = (orc_hist *)calloc(1, sizeof(orc_hist));
    return h;
}

void orc_history_free(void *hp)
{
    orc_hist *h = (orc_hist *)hp;
    if (!h) return;
    free(h->i); free(h->j); free(h->ut); free(h->age); free(h->wc); free(h);
}

int64_t orc_history_size(const void *hp) { return hp ? ((const orc_hist *)hp)->n : 0; }

static int hist_reserve(orc_hist *h, int64_t n)
{
    if (n <= h->cap) return 0;
    int64_t c = h->cap ? h->cap : 64;
    while (c < n) c *= 2;
    int64_t *ni = (int64_t *)realloc(h->i, (size_t)c * sizeof(int64_t));
    if (!ni) return ORC_ERR_NOMEM;
    h->i = ni;
    int64_t *nj = (int64_t *)realloc(h->j, (size_t)c * sizeof(int64_t));
    if (!nj) return ORC_ERR_NOMEM;
    h->j = nj;
    double *nu = (double *)realloc(h->ut, (size_t)c * 3 * sizeof(double));
    if (!nu) return ORC_ERR_NOMEM;
    h->ut = nu;
    double *na = (double *)realloc(h->age, (size_t)c * sizeof(double));
    if (!na) return ORC_ERR_NOMEM;
    h->age = na;
    double *nw = (double *)realloc(h->wc, (size_t)c * 4 * sizeof(double));
    if (!nw) return ORC_ERR_NOMEM;
    h->wc = nw;
    h->cap = c;
    return 0;
}

/* Binary search; returns the entry index or -1. */
static int64_t hist_find(const orc_hist *h, int64_t i, int64_t j)
{
    int64_t lo = 0, hi = h->n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (key_less(h->i[mid], h->j[mid], i, j)) lo = mid + 1;
        else hi = mid;
    }
    if (lo < h->n && h->i[lo] == i && h->j[lo] == j) return lo;
    return -1;
}

typedef struct { int64_t i, j, k; } hist_ref;

static int hist_ref_cmp(const void *a, const void *b)
{
    const hist_ref *x = (const hist_ref *)a, *y = (const hist_ref *)b;
    if (key_less(x->i, x->j, y->i, y->j)) return -1;
    if (key_less(y->i, y->j, x->i, x->j)) return 1;
    return x->k < y->k ? -1 : (x->k > y->k ? 1 : 0);
}

int orc_history_set(void *hp, int64_t n, const int64_t *i, const int64_t *j, const double *ut, const double *age)
{
    orc_hist *h = (orc_hist *)hp;
    if (!h || n < 0) return ORC_ERR_ARG;
    if (hist_reserve(h, n)) return ORC_ERR_NOMEM;
    /* entries sorted by (i, partner) for hist_find */
    hist_ref *r = (hist_ref *)malloc((size_t)(n > 0 ? n : 1) * sizeof(hist_ref));
    if (!r) return ORC_ERR_NOMEM;
    for (int64_t k = 0; k < n; ++k) { r[k].i = i[k]; r[k].j = j[k]; r[k].k = k; }
    qsort(r, (size_t)n, sizeof(hist_ref), hist_ref_cmp);
    for (int64_t k = 0; k < n; ++k) {
        h->i[k] = r[k].i; h->j[k] = r[k].j;
        memcpy(&h->ut[3 * k], &ut[3 * r[k].k], 3 * sizeof(double));
        h->age[k] = age ? age[r[k].k] : 0.0;
        h->wc[4 * k] = h->wc[4 * k + 1] = h->wc[4 * k + 2] = h->wc[4 * k + 3] = 0.0;
    }
    h->n = n;
    free(r);
    return 0;
}

int orc_history_set_wildcards(void *hp, int64_t n, const int64_t *i, const int64_t *j, const double *wc)
{
    orc_hist *h = (orc_hist *)hp;
    if (!h || n < 0) return ORC_ERR_ARG;
    /* entries not present are added with zero history, then the whole set re-sorted */
    int64_t n0 = h->n, add = 0;
    for (int64_t k = 0; k < n; ++k)
        if (hist_find(h, i[k], j[k]) < 0) ++add;
    if (add) {
        int64_t tot = n0 + add;
        int64_t *ni = (int64_t *)malloc((size_t)tot * sizeof(int64_t));
        int64_t *nj = (int64_t *)malloc((size_t)tot * sizeof(int64_t));
        double *nu = (double *)malloc((size_t)tot * 3 * sizeof(double));
        double *na = (double *)malloc((size_t)tot * sizeof(double));
        double *nw = (double *)malloc((size_t)tot * 4 * sizeof(double));
        if (!ni || !nj || !nu || !na || !nw) { free(ni); free(nj); free(nu); free(na); free(nw); return ORC_ERR_NOMEM; }
        memcpy(ni, h->i, (size_t)n0 * sizeof(int64_t));
        memcpy(nj, h->j, (size_t)n0 * sizeof(int64_t));
        memcpy(nu, h->ut, (size_t)n0 * 3 * sizeof(double));
        memcpy(na, h->age, (size_t)n0 * sizeof(double));
        memcpy(nw, h->wc, (size_t)n0 * 4 * sizeof(double));
        int64_t m = n0;
        for (int64_t k = 0; k < n; ++k) {
            if (hist_find(h, i[k], j[k]) >= 0) continue;
            ni[m] = i[k]; nj[m] = j[k];
            nu[3 * m] = nu[3 * m + 1] = nu[3 * m + 2] = 0.0;
            na[m] = 0.0;
            nw[4 * m] = nw[4 * m + 1] = nw[4 * m + 2] = nw[4 * m + 3] = 0.0;
            ++m;
        }
        int e = orc_history_set(h, tot, ni, nj, nu, na);
        /* orc_history_set cleared the wildcards: put the kept ones back */
        for (int64_t k = 0; k < tot && !e; ++k) {
            int64_t q = hist_find(h, ni[k], nj[k]);
            memcpy(&h->wc[4 * q], &nw[4 * k], 4 * sizeof(double));
        }
        free(ni); free(nj); free(nu); free(na); free(nw);
        if (e) return e;
    }
    for (int64_t k = 0; k < n; ++k) {
        int64_t q = hist_find(h, i[k], j[k]);
        memcpy(&h->wc[4 * q], &wc[4 * k], 4 * sizeof(double));
    }
    return 0;
}

int orc_history_get_wildcards(const void *hp, int64_t cap, int64_t *n, double *wc)
{
    const orc_hist *h = (const orc_hist *)hp;
    if (!h) return ORC_ERR_ARG;
    *n = h->n;
    if (h->n > cap) return ORC_ERR_CAPACITY;
    memcpy(wc, h->wc, (size_t)h->n * 4 * sizeof(double));
    return 0;
}

int orc_history_get(const void *hp, int64_t cap, int64_t *n, int64_t *i, int64_t *j, double *ut, double *age)
{
    const orc_hist *h = (const orc_hist *)hp;
    if (!h) return ORC_ERR_ARG;
    *n = h->n;
    if (h->n > cap) return ORC_ERR_CAPACITY;
    for (int64_t k = 0; k < h->n; ++k) {
        i[k] = h->i[k]; j[k] = h->j[k];
        ut[3 * k] = h->ut[3 * k]; ut[3 * k + 1] = h->ut[3 * k + 1]; ut[3 * k + 2] = h->ut[3 * k + 2];
        if (age) age[k] = h->age[k];
    }
    return 0;
}

/* ------------------------------------------------------------------ geometry */

int orc_sphere_positions(const orc_world *w, double *p)
{
    const int nt = w->n_threads > 1 ? w->n_threads : 1;
    (void)nt;
#pragma omp parallel for num_threads(nt) if (nt > 1) schedule(static)
    for (int64_t s = 0; s < w->n_sphere; ++s) {
        int64_t o = w->owner[s];
        double R[9], r[3];
        quat_matrix(&w->q[4 * o], R);
        mat_vec(R, &w->rloc[3 * s], r);
        p[3 * s + 0] = w->x[3 * o + 0] + r[0];
        p[3 * s + 1] = w->x[3 * o + 1] + r[1];
        p[3 * s + 2] = w->x[3 * o + 2] + r[2];
    }
    return 0;
}

/* Point of the triangle (a, b, c) closest to p: the region tests of the published
 * closest-point-on-triangle algorithm (vertex, edge and face regions by the signs of
 * barycentric-coordinate numerators), evaluated in this order. */
static void closest_on_triangle(const double p[3], const double a[3], const double b[3], const double c[3],
                                double q[3])
{
    double ab[3], ac[3], ap[3], bp[3], cp[3];
    for (int k = 0; k < 3; ++k) {
        ab[k] = b[k] - a[k]; ac[k] = c[k] - a[k]; ap[k] = p[k] - a[k];
        bp[k] = p[k] - b[k]; cp[k] = p[k] - c[k];
    }
    double d1 = dot3(ab, ap), d2 = dot3(ac, ap);
    if (d1 <= 0.0 && d2 <= 0.0) { memcpy(q, a, 3 * sizeof(double)); return; }
    double d3 = dot3(ab, bp), d4 = dot3(ac, bp);
    if (d3 >= 0.0 && d4 <= d3) { memcpy(q, b, 3 * sizeof(double)); return; }
    double vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
        double v = d1 / (d1 - d3);
        for (int k = 0; k < 3; ++k) q[k] = a[k] + v * ab[k];
        return;
    }
    double d5 = dot3(ab, cp), d6 = dot3(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) { memcpy(q, c, 3 * sizeof(double)); return; }
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
        double w = d2 / (d2 - d6);
        for (int k = 0; k < 3; ++k) q[k] = a[k] + w * ac[k];
        return;
    }
    double va = d3 * d6 - d5 * d4;
    if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) {
        double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        for (int k = 0; k < 3; ++k) q[k] = b[k] + w * (c[k] - b[k]);
        return;
    }
    double den = 1.0 / ((va + vb) + vc);
    double v = vb * den, w = vc * den;
    for (int k = 0; k < 3; ++k) q[k] = (a[k] + ab[k] * v) + ac[k] * w;
}

/* Vertices of a facet wall at time t: p + R(omega t)(v - p) (Rodrigues' rotation about
 * the unit axis omega / |omega| by |omega| t). */
static void facet_vertices(const orc_wall *wl, double t, double v[9])
{
    double wn = norm3(wl->omega);
    if (!(wn > 0.0)) { memcpy(v, wl->tri, 9 * sizeof(double)); return; }
    double k[3] = {wl->omega[0] / wn, wl->omega[1] / wn, wl->omega[2] / wn};
    double th = wn * t, cs = cos(th), sn = sin(th);
    for (int m = 0; m < 3; ++m) {
        double r[3] = {wl->tri[3 * m] - wl->p[0], wl->tri[3 * m + 1] - wl->p[1], wl->tri[3 * m + 2] - wl->p[2]};
        double kxr[3];
        cross3(k, r, kxr);
        double kr = dot3(k, r);
        for (int a = 0; a < 3; ++a)
            v[3 * m + a] = wl->p[a] + ((r[a] * cs + kxr[a] * sn) + k[a] * (kr * (1.0 - cs)));
    }
}

/* Signed gap from a sphere centre c to a wall surface (positive on the domain side)
 * and the unit normal from the wall towards the centre.  Returns 0 if the normal is
 * undefined (centre on a cylinder or cone axis), 1 otherwise. */
static int wall_gap(const orc_wall *wl, double tnow, const double c[3], double *gap, double nrm[3])
{
    const double *a = wl->p, *u = wl->n;
    double d[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    if (wl->type == ORC_WALL_TRIANGLE) {
        /* two-sided facet at time t: distance to its closest point */
        double v[9], q[3];
        facet_vertices(wl, tnow, v);
        closest_on_triangle(c, &v[0], &v[3], &v[6], q);
        double e[3] = {c[0] - q[0], c[1] - q[1], c[2] - q[2]};
        double dist = norm3(e);
        *gap = dist;
        if (!(dist > 0.0)) return 0;
        nrm[0] = e[0] / dist; nrm[1] = e[1] / dist; nrm[2] = e[2] / dist;
        return 1;
    }
    if (wl->type == ORC_WALL_PLANE) {
        *gap = (d[0] * u[0] + d[1] * u[1]) + d[2] * u[2];
        nrm[0] = u[0]; nrm[1] = u[1]; nrm[2] = u[2];
        return 1;
    }
    double z = (d[0] * u[0] + d[1] * u[1]) + d[2] * u[2];
    double rp[3] = {d[0] - z * u[0], d[1] - z * u[1], d[2] - z * u[2]};
    double rho = sqrt((rp[0] * rp[0] + rp[1] * rp[1]) + rp[2] * rp[2]);
    if (wl->type == ORC_WALL_CYLINDER) {
        *gap = wl->r0 - rho;
        if (!(rho > 0.0)) return 0;
        nrm[0] = -rp[0] / rho; nrm[1] = -rp[1] / rho; nrm[2] = -rp[2] / rho;
        return 1;
    }
    /* cone segment: closest point of the generator segment in the (rho, z) half plane */
    double dr = wl->r1 - wl->r0, dz = wl->z1 - wl->z0;
    double len2 = dr * dr + dz * dz;
    double t = ((rho - wl->r0) * dr + (z - wl->z0) * dz) / len2;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    double cr = wl->r0 + t * dr, cz = wl->z0 + t * dz;
    double Dr = rho - cr, Dz = z - cz;
    double dist = sqrt(Dr * Dr + Dz * Dz);
    /* inward normal of the generator line: the one with a negative radial part */
    double len = sqrt(len2);
    double inr = -dz / len, inz = dr / len;
    if (inr > 0.0) { inr = -inr; inz = -inz; }
    double side = Dr * inr + Dz * inz;
    double sgn = side >= 0.0 ? 1.0 : -1.0;
    *gap = sgn * dist;
    if (!(rho > 0.0) || !(dist > 0.0)) return 0;
    double n2r = sgn * Dr / dist, n2z = sgn * Dz / dist;
    double er[3] = {rp[0] / rho, rp[1] / rho, rp[2] / rho};
    nrm[0] = n2r * er[0] + n2z * u[0];
    nrm[1] = n2r * er[1] + n2z * u[1];
    nrm[2] = n2r * er[2] + n2z * u[2];
    return 1;
}

static int owner_is_active(const orc_world *w, int64_t o) { return w->active ? w->active[o] != 0 : 1; }

static int owner_family(const orc_world *w, int64_t o) { return w->family ? (int)w->family[o] : 0; }

/* Contacts between owners a and b are resolved (the families' contact mask). */
static int families_meet(const orc_world *w, int64_t a, int64_t b)
{
    if (!w->contact_mask) return 1;
    return w->contact_mask[owner_family(w, a) * 256 + owner_family(w, b)] != 0;
}

/* Threads of the parallel loops (1 = serial). */
static int n_threads(const orc_world *w) { return w->n_threads > 1 ? w->n_threads : 1; }

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int orc_listed_pairs_f64(int64_t n, const double *p, const double *rad, const int64_t *owner,
                         const uint8_t *sphere_active, double beta, int64_t cap,
                         int64_t *count, int64_t *pi, int64_t *pj)
{
    int64_t c = 0;
    double b2 = 2.0 * beta;
    for (int64_t i = 0; i < n; ++i) {
        if (sphere_active && !sphere_active[i]) continue;
        for (int64_t j = i + 1; j < n; ++j) {
            if (sphere_active && !sphere_active[j]) continue;
            if (owner[i] == owner[j]) continue;
            double dx = p[3 * i + 0] - p[3 * j + 0];
            double dy = p[3 * i + 1] - p[3 * j + 1];
            double dz = p[3 * i + 2] - p[3 * j + 2];
            double s = (dx * dx + dy * dy) + dz * dz;
            double t = (rad[i] + rad[j]) + b2;
            if (s < t * t) {
                if (c < cap) { pi[c] = i; pj[c] = j; }
                ++c;
            }
        }
    }
    *count = c;
    return c > cap ? ORC_ERR_CAPACITY : 0;
}

int orc_listed_pairs_voxel_f32(int64_t n, const int32_t *cell, const float *off, float L,
                               const float *rad, const int64_t *owner,
                               const uint8_t *sphere_active, float beta, int64_t cap,
                               int64_t *count, int64_t *pi, int64_t *pj)
{
    int64_t c = 0;
    float b2 = 2.0f * beta;
    for (int64_t i = 0; i < n; ++i) {
        if (sphere_active && !sphere_active[i]) continue;
        for (int64_t j = i + 1; j < n; ++j) {
            if (sphere_active && !sphere_active[j]) continue;
            if (owner[i] == owner[j]) continue;
            float d[3];
            for (int k = 0; k < 3; ++k) {
                float dc = (float)(cell[3 * i + k] - cell[3 * j + k]);
                float doff = off[3 * i + k] - off[3 * j + k];
                float cl = dc * L;
                d[k] = cl + doff;
            }
            float s = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            float t = (rad[i] + rad[j]) + b2;
            if (s < t * t) {
                if (c < cap) { pi[c] = i; pj[c] = j; }
                ++c;
            }
        }
    }
    *count = c;
    return c > cap ? ORC_ERR_CAPACITY : 0;
}

int orc_listed_wall_pairs(const orc_world *w, const double *p, double beta, int64_t cap,
                          int64_t *count, int64_t *si, int64_t *wi)
{
    int64_t c = 0;
    for (int64_t s = 0; s < w->n_sphere; ++s) {
        if (!owner_is_active(w, w->owner[s])) continue;
        for (int32_t k = 0; k < w->n_wall; ++k) {
            double gap, nrm[3];
            wall_gap(&w->walls[k], (double)w->step * w->h, &p[3 * s], &gap, nrm);
            if (gap < w->rad[s] + beta) {
                if (c < cap) { si[c] = s; wi[c] = k; }
                ++c;
            }
        }
    }
    *count = c;
    return c > cap ? ORC_ERR_CAPACITY : 0;
}

/* ------------------------------------------------------------------ contact force */

/* Kinematic inputs of one contact: A is a sphere; B is a sphere or a wall. */
typedef struct {
    double n[3];       /* unit normal from B to A */
    double delta;      /* overlap, > 0 */
    double c[3];       /* contact point */
    double uA[3];      /* velocity of the contact point as a point of A */
    double uB[3];      /* ... as a point of B */
    double rotA[3];    /* the rotational part of uA: (angular velocity of A) x (c - x_A) */
    double rotB[3];    /* ... of uB (for a wall its whole surface velocity) */
    double Rbar, mbar;
    double Estar, Gstar, beta, mu, crr;
    double RA, RB;     /* radii of the two geometries (a wall: 0) */
    double nu;         /* mean of the two materials' Poisson ratios */
} contact_in;

/* Whether a contact that has lasted `age` is still inside its first collision: the
 * default model of Sec. 4.2.1 applies rolling resistance only after a collision time of
 * a damped linear oscillator, whose stiffness and damping it forms from E*, the damping
 * ratio and the effective mass and radius in a simplified way.  This follows that
 * reading term by term: with s = sqrt(Rbar), k = (4/3) E* sqrt(s) and
 * g = -2 sqrt((5/3) mbar E*) beta s^(1/4), the damping ratio is z = g / (2 sqrt(k mbar))
 * and, where z < 1 and 1 - z^2 > 0, the collision time is pi sqrt(mbar / (k (1 - z^2))). */
static int within_collision_time(const contact_in *ci, double age)
{
    double s = sqrt(ci->Rbar);
    double k = (4.0 / 3.0) * ci->Estar * sqrt(s);
    double g = -2.0 * sqrt((5.0 / 3.0) * ci->mbar * ci->Estar) * ci->beta * sqrt(sqrt(s));
    double z = g / (2.0 * sqrt(k * ci->mbar));
    if (!(z < 1.0)) return 0;
    double d = 1.0 - z * z;
    if (!(d > 0.0)) return 0;
    double tc = ORC_PI * sqrt(ci->mbar / (k * d));
    return age <= tc;
}

/* The default history-based Hertz-Mindlin model (Sec. 4.1 Eqs. 1-4 as the listing of
 * Sec. 4.2.1 computes it), with rolling resistance.  ut and age (time in contact) are
 * updated in place; F is the force on A; Fr the rolling-resistance force on A, which
 * acts only through the contact torque (B receives -Fr). */
static void hertz_mindlin(const contact_in *ci, double h, double ut[3], double *age, double F[3], double Fr[3])
{
    const double *n = ci->n;
    double u[3] = {ci->uA[0] - ci->uB[0], ci->uA[1] - ci->uB[1], ci->uA[2] - ci->uB[2]};
    double proj = dot3(u, n);
    double vt[3] = {u[0] - proj * n[0], u[1] - proj * n[1], u[2] - proj * n[2]};

    /* history update precedes the force: accumulate h*vt, then remove the normal part;
     * the contact's age grows by h */
    ut[0] = ut[0] + h * vt[0];
    ut[1] = ut[1] + h * vt[1];
    ut[2] = ut[2] + h * vt[2];
    double up = dot3(ut, n);
    ut[0] = ut[0] - up * n[0];
    ut[1] = ut[1] - up * n[1];
    ut[2] = ut[2] - up * n[2];
    *age = *age + h;

    double c56 = sqrt(5.0 / 6.0);
    double sqrtRd = sqrt(ci->delta * ci->Rbar);
    double Sn = 2.0 * ci->Estar * sqrtRd;
    double kn = (2.0 / 3.0) * Sn;
    double gn = 2.0 * c56 * ci->beta * sqrt(Sn * ci->mbar);
    double fn = kn * ci->delta + gn * proj;
    F[0] = fn * n[0]; F[1] = fn * n[1]; F[2] = fn * n[2];

    /* rolling resistance: C_r times the normal force (damping included), along the
     * rolling part of B's contact-point velocity relative to A's, once the contact has
     * outlasted its collision time */
    Fr[0] = 0.0; Fr[1] = 0.0; Fr[2] = 0.0;
    if (ci->crr > 0.0 && !within_collision_time(ci, *age)) {
        double vr[3] = {ci->rotB[0] - ci->rotA[0], ci->rotB[1] - ci->rotA[1], ci->rotB[2] - ci->rotA[2]};
        double vm = norm3(vr);
        if (vm > 1e-12) {
            double sc = ci->crr * norm3(F) / vm;
            Fr[0] = sc * vr[0]; Fr[1] = sc * vr[1]; Fr[2] = sc * vr[2];
        }
    }

    if (ci->mu > 0.0) {
        double kt = 8.0 * ci->Gstar * sqrtRd;
        double gt = -2.0 * c56 * ci->beta * sqrt(ci->mbar * kt);
        double Ft[3] = {-kt * ut[0] - gt * vt[0], -kt * ut[1] - gt * vt[1], -kt * ut[2] - gt * vt[2]};
        double ft = norm3(Ft);
        if (ft > 1e-12) {
            double ftmax = norm3(F) * ci->mu;
            if (ft > ftmax) {
                double sc = ftmax / ft;
                Ft[0] = sc * Ft[0]; Ft[1] = sc * Ft[1]; Ft[2] = sc * Ft[2];
                ut[0] = (Ft[0] + gt * vt[0]) / (-kt);
                ut[1] = (Ft[1] + gt * vt[1]) / (-kt);
                ut[2] = (Ft[2] + gt * vt[2]) / (-kt);
            }
        } else {
            Ft[0] = 0.0; Ft[1] = 0.0; Ft[2] = 0.0;
        }
        F[0] = F[0] + Ft[0]; F[1] = F[1] + Ft[1]; F[2] = F[2] + Ft[2];
    }
}

/* The bonded, breakable contact of Sec. 6.3 (the paper's worked custom model, after the
 * constitutive laws it cites), for a bonded pair (wc[0] > 1e-12; wc[1] is the overlap at
 * which the bond carries no load).  The readings of the partial listing are those of the
 * equations printed beside it:
 *   D = delta - wc[1], k_n = E* Rbar, area A = pi max(R_A, R_B)^2, bond strength
 *   F_b = sigma_t A (sigma_t < 0: tension), D_y = F_b / k_n, D_u = 3 D_y;
 *   normal force k_n D above D_y, softening linearly to zero at D_u below it (the
 *   printed equation's slope -k_n / xi with xi = 2, continuous at D_y), damped by
 *   0.01 sqrt(mbar k_n) times the normal relative velocity; the bond breaks
 *   (wc[0] = -1) once D < D_u;
 *   tangential: the history update of the default model, k_t = nu k_n (nu the mean of
 *   the two materials'), damping g_t = -2 sqrt(5/6) beta sqrt(mbar k_t) opposing sliding
 *   as in the default model, F_t = -k_t ut - g_t v_t; the bond breaks once |F_t|
 *   exceeds mu |F| + c A (c the cohesion; c A only while D > D_y);
 *   bending: a torque-only force of magnitude min(h R_A R_B k_t / R_A, eta |F|) along the
 *   rolling part of B's contact-point velocity relative to A's (as rolling resistance).
 * A is the lower sphere id (the bending term is not symmetric in A and B). */
static void bonded_breakage(const contact_in *ci, const double *par, double h, double ut[3], double *age,
                            double wc[4], double F[3], double Fr[3])
{
    const double *n = ci->n;
    double u[3] = {ci->uA[0] - ci->uB[0], ci->uA[1] - ci->uB[1], ci->uA[2] - ci->uB[2]};
    double proj = dot3(u, n);
    double vt[3] = {u[0] - proj * n[0], u[1] - proj * n[1], u[2] - proj * n[2]};
    ut[0] = ut[0] + h * vt[0];
    ut[1] = ut[1] + h * vt[1];
    ut[2] = ut[2] + h * vt[2];
    double up = dot3(ut, n);
    ut[0] = ut[0] - up * n[0];
    ut[1] = ut[1] - up * n[1];
    ut[2] = ut[2] - up * n[2];
    *age = *age + h;

    double D = ci->delta - wc[1];
    double kn = ci->Estar * ci->Rbar;
    double Rm = ci->RA > ci->RB ? ci->RA : ci->RB;
    double area = ORC_PI * (Rm * Rm);
    double Dy = (par[ORC_BRK_TENSION] * area) / kn;
    double Du = 3.0 * Dy;
    double fn = D > Dy ? kn * D : 0.5 * kn * (Du - D);
    double gn = par[ORC_BRK_DAMPING] * sqrt(ci->mbar * kn);
    double fnd = fn - gn * proj;
    F[0] = fnd * n[0]; F[1] = fnd * n[1]; F[2] = fnd * n[2];
    if (D < Du) wc[0] = -1.0;

    double kt = ci->nu * kn;
    double c56 = sqrt(5.0 / 6.0);
    double gt = -2.0 * c56 * ci->beta * sqrt(ci->mbar * kt);
    double fs_max = norm3(F) * ci->mu + (D > Dy ? par[ORC_BRK_COHESION] * area : 0.0);
    double Ft[3] = {-kt * ut[0] - gt * vt[0], -kt * ut[1] - gt * vt[1], -kt * ut[2] - gt * vt[2]};
    if (norm3(Ft) > fs_max) wc[0] = -1.0;
    F[0] = F[0] + Ft[0]; F[1] = F[1] + Ft[1]; F[2] = F[2] + Ft[2];

    Fr[0] = 0.0; Fr[1] = 0.0; Fr[2] = 0.0;
    double vr[3] = {ci->rotB[0] - ci->rotA[0], ci->rotB[1] - ci->rotA[1], ci->rotB[2] - ci->rotA[2]};
    double vm = norm3(vr);
    if (vm > 1e-12) {
        double kr = (ci->RA * ci->RB) * kt;
        double m1 = (h * kr) / ci->RA, m2 = par[ORC_BRK_ETA] * norm3(F);
        double sc = (m1 < m2 ? m1 : m2) / vm;
        Fr[0] = sc * vr[0]; Fr[1] = sc * vr[1]; Fr[2] = sc * vr[2];
    }
}

/* Velocity of a point `c` carried by owner o: v + (R(q) wb) x (c - x); rot receives
 * the rotational part (R(q) wb) x (c - x). */
static void owner_point_velocity(const orc_world *w, int64_t o, const double c[3], double out[3], double rot[3])
{
    double R[9], wg[3], r[3];
    quat_matrix(&w->q[4 * o], R);
    mat_vec(R, &w->wb[3 * o], wg);
    r[0] = c[0] - w->x[3 * o + 0]; r[1] = c[1] - w->x[3 * o + 1]; r[2] = c[2] - w->x[3 * o + 2];
    cross3(wg, r, rot);
    out[0] = w->v[3 * o + 0] + rot[0];
    out[1] = w->v[3 * o + 1] + rot[1];
    out[2] = w->v[3 * o + 2] + rot[2];
}

/* Fill the pair-dependent material part of a contact. */
static void contact_material(const orc_world *w, int32_t ma, int32_t mb, contact_in *ci)
{
    orc_effective_moduli(w->E[ma], w->nu[ma], w->E[mb], w->nu[mb], &ci->Estar, &ci->Gstar);
    ci->beta = damping_beta(w->cor[ma * w->n_mat + mb]);
    ci->mu = w->mu[ma * w->n_mat + mb];
    ci->crr = w->crr ? w->crr[ma * w->n_mat + mb] : 0.0;
    ci->nu = 0.5 * (w->nu[ma] + w->nu[mb]);
}

/* Geometry of the sphere pair (A = i, B = j) whatever the sign of the overlap (a bonded
 * contact acts in tension too).  Returns 0 only where the centres coincide. */
static int sphere_pair_geometry(const orc_world *w, const double *p, int64_t i, int64_t j, contact_in *ci)
{
    double dx[3] = {p[3 * i + 0] - p[3 * j + 0], p[3 * i + 1] - p[3 * j + 1], p[3 * i + 2] - p[3 * j + 2]};
    double d = sqrt((dx[0] * dx[0] + dx[1] * dx[1]) + dx[2] * dx[2]);
    double RA = w->rad[i], RB = w->rad[j];
    double delta = (RA + RB) - d;
    if (!(d > 0.0)) return 0;
    ci->RA = RA; ci->RB = RB;
    double inv = 1.0 / d;
    ci->n[0] = dx[0] * inv; ci->n[1] = dx[1] * inv; ci->n[2] = dx[2] * inv;
    ci->delta = delta;
    /* contact point: midpoint of the overlap segment along the normal */
    double a = RA - 0.5 * delta;
    ci->c[0] = p[3 * i + 0] - a * ci->n[0];
    ci->c[1] = p[3 * i + 1] - a * ci->n[1];
    ci->c[2] = p[3 * i + 2] - a * ci->n[2];
    int64_t oa = w->owner[i], ob = w->owner[j];
    owner_point_velocity(w, oa, ci->c, ci->uA, ci->rotA);
    owner_point_velocity(w, ob, ci->c, ci->uB, ci->rotB);
    ci->Rbar = (RA * RB) / (RA + RB);
    ci->mbar = (w->mass[oa] * w->mass[ob]) / (w->mass[oa] + w->mass[ob]);
    contact_material(w, w->mat[i], w->mat[j], ci);
    return 1;
}

/* The same where the spheres touch: returns 1 iff delta > 0. */
static int sphere_pair_contact(const orc_world *w, const double *p, int64_t i, int64_t j, contact_in *ci)
{
    return sphere_pair_geometry(w, p, i, j, ci) && ci->delta > 0.0;
}

/* Geometry of sphere i against wall k (A = sphere, B = wall: infinite radius and mass). */
static int sphere_wall_contact(const orc_world *w, const double *p, int64_t i, int32_t k, contact_in *ci)
{
    const orc_wall *wl = &w->walls[k];
    double gap, nrm[3];
    if (!wall_gap(wl, (double)w->step * w->h, &p[3 * i], &gap, nrm)) return 0;
    double RA = w->rad[i];
    double delta = RA - gap;
    if (!(delta > 0.0)) return 0;
    ci->n[0] = nrm[0]; ci->n[1] = nrm[1]; ci->n[2] = nrm[2];
    ci->delta = delta;
    double a = RA - 0.5 * delta;
    ci->c[0] = p[3 * i + 0] - a * nrm[0];
    ci->c[1] = p[3 * i + 1] - a * nrm[1];
    ci->c[2] = p[3 * i + 2] - a * nrm[2];
    int64_t oa = w->owner[i];
    owner_point_velocity(w, oa, ci->c, ci->uA, ci->rotA);
    double r[3] = {ci->c[0] - wl->p[0], ci->c[1] - wl->p[1], ci->c[2] - wl->p[2]};
    cross3(wl->omega, r, ci->uB);
    memcpy(ci->rotB, ci->uB, sizeof(ci->uB));   /* a wall moves by rotation only */
    ci->Rbar = RA;
    ci->mbar = w->mass[oa];
    ci->RA = RA; ci->RB = 0.0;
    contact_material(w, w->mat[i], wl->mat, ci);
    return 1;
}

/* ------------------------------------------------------------------ one evaluation */

typedef struct {
    int64_t n, cap;
    orc_contact *c;
} contact_buf;

static int cbuf_push(contact_buf *b, const orc_contact *c)
{
    if (b->n == b->cap) {
        int64_t nc = b->cap ? 2 * b->cap : 256;
        orc_contact *nb = (orc_contact *)realloc(b->c, (size_t)nc * sizeof(orc_contact));
        if (!nb) return ORC_ERR_NOMEM;
        b->c = nb; b->cap = nc;
    }
    b->c[b->n++] = *c;
    return 0;
}

/* One candidate partner jj of sphere i (a sphere when jj < N, else wall jj - N): if the
 * two touch, the contact with its force and updated history in *rec; returns 1 then. */
static int contact_of(const orc_world *w, const double *p, const orc_hist *h, int64_t i, int64_t jj,
                      orc_contact *rec)
{
    int64_t N = w->n_sphere;
    int64_t oa = w->owner[i];
    contact_in ci;
    int64_t j;
    int bonded = 0;
    if (jj < N) {
        j = jj;
        int64_t ob = w->owner[j];
        if (ob == oa || !owner_is_active(w, ob) || !families_meet(w, oa, ob)) return 0;
        if (w->model == ORC_MODEL_BONDED_BREAKAGE) {
            /* a bonded pair acts whatever the sign of its overlap */
            int64_t hb = h ? hist_find(h, i, j) : -1;
            bonded = hb >= 0 && h->wc[4 * hb] > 1e-12;
        }
        if (bonded ? !sphere_pair_geometry(w, p, i, j, &ci) : !sphere_pair_contact(w, p, i, j, &ci)) return 0;
    } else {
        int32_t k = (int32_t)(jj - N);
        j = -1 - (int64_t)k;
        if (!sphere_wall_contact(w, p, i, k, &ci)) return 0;
    }
    memset(rec, 0, sizeof(*rec));
    rec->i = i; rec->j = j;
    int64_t hk = h ? hist_find(h, i, j) : -1;
    if (hk >= 0) {
        rec->ut[0] = h->ut[3 * hk]; rec->ut[1] = h->ut[3 * hk + 1]; rec->ut[2] = h->ut[3 * hk + 2];
        rec->age = h->age[hk];
        memcpy(rec->wc, &h->wc[4 * hk], sizeof(rec->wc));
    }
    if (bonded)
        bonded_breakage(&ci, w->model_params, w->h, rec->ut, &rec->age, rec->wc, rec->force, rec->torque_force);
    else
        hertz_mindlin(&ci, w->h, rec->ut, &rec->age, rec->force, rec->torque_force);
    memcpy(rec->point, ci.c, sizeof(ci.c));
    memcpy(rec->normal, ci.n, sizeof(ci.n));
    rec->overlap = ci.delta;
    return 1;
}

/* Reduction of one contact onto the owners (Eqs. 5a-5b): F on A's owner, -F on B's;
 * torques about the centres of mass. */
static void add_to_owners(const orc_world *w, const orc_contact *rec, double *F, double *T)
{
    int64_t oa = w->owner[rec->i];
    double rA[3] = {rec->point[0] - w->x[3 * oa], rec->point[1] - w->x[3 * oa + 1], rec->point[2] - w->x[3 * oa + 2]};
    double tA[3], rrA[3];
    cross3(rA, rec->force, tA);
    cross3(rA, rec->torque_force, rrA);
    for (int k = 0; k < 3; ++k) {
        F[3 * oa + k] += rec->force[k];
        T[3 * oa + k] += tA[k];
        T[3 * oa + k] += rrA[k];
    }
    if (rec->j >= 0) {
        int64_t ob = w->owner[rec->j];
        double rB[3] = {rec->point[0] - w->x[3 * ob], rec->point[1] - w->x[3 * ob + 1], rec->point[2] - w->x[3 * ob + 2]};
        double mf[3] = {-rec->force[0], -rec->force[1], -rec->force[2]};
        double mr[3] = {-rec->torque_force[0], -rec->torque_force[1], -rec->torque_force[2]};
        double tB[3], rrB[3];
        cross3(rB, mf, tB);
        cross3(rB, mr, rrB);
        for (int k = 0; k < 3; ++k) {
            F[3 * ob + k] += mf[k];
            T[3 * ob + k] += tB[k];
            T[3 * ob + k] += rrB[k];
        }
    }
}

/* ------------------------------------------------------------------ optional grid
 * A faster way to enumerate the same candidates (cell_list = 1).  Spheres of active
 * owners are binned into cubes of edge 2 r_max (1 + 1e-6): two spheres that touch are
 * less than r_i + r_j <= 2 r_max apart, so they sit in the same or adjacent cubes.  The
 * candidates j > i of the 27 cubes around sphere i are sorted ascending and visited in
 * that order, so the contacts, their order and every floating-point sum equal those of
 * the plain loop over all j > i (a test checks trajectories bit for bit).  Positions
 * that are not finite, or too far apart for 64-bit cube indices, fall back to the plain
 * loop. */
typedef struct { int64_t c[3]; int64_t idx; } grid_ent;

static int grid_ent_cmp(const void *a, const void *b)
{
    const grid_ent *x = (const grid_ent *)a, *y = (const grid_ent *)b;
    for (int k = 0; k < 3; ++k) {
        if (x->c[k] != y->c[k]) return x->c[k] < y->c[k] ? -1 : 1;
    }
    return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0);
}

static int i64_cmp(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* first entry whose cube is not below c (entries sorted by grid_ent_cmp) */
static int64_t grid_lower(const grid_ent *e, int64_t n, const int64_t c[3])
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int below = 0;
        for (int k = 0; k < 3; ++k) {
            if (e[mid].c[k] != c[k]) { below = e[mid].c[k] < c[k]; break; }
        }
        if (below) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* Bins the spheres of active owners; returns 1 with *out (sorted, n entries, caller
 * frees) on success, 0 when the plain loop must be used, or a negative error. */
static int grid_build(const orc_world *w, const double *p, grid_ent **out, int64_t *n_out, int64_t **home_out)
{
    int64_t N = w->n_sphere;
    double rmax = 0.0;
    for (int64_t s = 0; s < N; ++s) rmax = w->rad[s] > rmax ? w->rad[s] : rmax;
    if (!(rmax > 0.0)) return 0;
    double cube = 2.0 * rmax * (1.0 + 1e-6);
    double lo[3] = {0.0, 0.0, 0.0};
    int any = 0;
    for (int64_t s = 0; s < N; ++s) {
        if (!owner_is_active(w, w->owner[s])) continue;
        for (int k = 0; k < 3; ++k) {
            double v = p[3 * s + k];
            if (!isfinite(v)) return 0;
            if (!any || v < lo[k]) lo[k] = v;
        }
        any = 1;
    }
    grid_ent *e = (grid_ent *)malloc((size_t)(N > 0 ? N : 1) * sizeof(grid_ent));
    int64_t *home = (int64_t *)malloc((size_t)(N > 0 ? N : 1) * 3 * sizeof(int64_t));
    if (!e || !home) { free(e); free(home); return ORC_ERR_NOMEM; }
    int64_t n = 0;
    for (int64_t s = 0; s < N; ++s) {
        if (!owner_is_active(w, w->owner[s])) continue;
        for (int k = 0; k < 3; ++k) {
            double u = floor((p[3 * s + k] - lo[k]) / cube);
            if (!(u >= 0.0 && u < 1e15)) { free(e); free(home); return 0; }
            e[n].c[k] = (int64_t)u;
            home[3 * s + k] = (int64_t)u;
        }
        e[n].idx = s;
        ++n;
    }
    qsort(e, (size_t)n, sizeof(grid_ent), grid_ent_cmp);
    *out = e;
    *n_out = n;
    *home_out = home;
    return 1;
}

/* Where each cube's entries start, when the cubes spanned are few (at most 8 per sphere
 * plus 4096): start[c] for the linear cube index c = (cx * ny + cy) * nz + cz, with
 * start[ncube] = n.  Returns NULL when the span is larger (binary search is used). */
static int64_t *grid_starts(const grid_ent *e, int64_t n, int64_t dims[3])
{
    int64_t span[3] = {0, 0, 0};
    for (int64_t a = 0; a < n; ++a)
        for (int k = 0; k < 3; ++k) span[k] = e[a].c[k] + 1 > span[k] ? e[a].c[k] + 1 : span[k];
    double cubes = (double)span[0] * (double)span[1] * (double)span[2];
    if (n == 0 || cubes > 8.0 * (double)n + 4096.0) return NULL;
    int64_t nc = span[0] * span[1] * span[2];
    int64_t *start = (int64_t *)malloc((size_t)(nc + 1) * sizeof(int64_t));
    if (!start) return NULL;
    int64_t a = 0;
    for (int64_t c = 0; c < nc; ++c) {
        start[c] = a;
        while (a < n && (e[a].c[0] * span[1] + e[a].c[1]) * span[2] + e[a].c[2] == c) ++a;
    }
    start[nc] = n;
    for (int k = 0; k < 3; ++k) dims[k] = span[k];
    return start;
}

/* The candidates j > i of the 27 cubes around sphere i, ascending; returns their number. */
static int64_t grid_candidates(const grid_ent *e, int64_t n, const int64_t *start, const int64_t dims[3],
                               const int64_t home[3], int64_t i, int64_t *cand)
{
    int64_t nc = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                int64_t c[3] = {home[0] + dx, home[1] + dy, home[2] + dz};
                int64_t a, b;
                if (start) {
                    if (c[0] < 0 || c[1] < 0 || c[2] < 0 || c[0] >= dims[0] || c[1] >= dims[1] || c[2] >= dims[2])
                        continue;
                    int64_t lin = (c[0] * dims[1] + c[1]) * dims[2] + c[2];
                    a = start[lin];
                    b = start[lin + 1];
                } else {
                    a = grid_lower(e, n, c);
                    b = n;
                }
                for (; a < b; ++a) {
                    if (e[a].c[0] != c[0] || e[a].c[1] != c[1] || e[a].c[2] != c[2]) break;
                    if (e[a].idx > i) cand[nc++] = e[a].idx;
                }
            }
    qsort(cand, (size_t)nc, sizeof(int64_t), i64_cmp);
    return nc;
}

/* Every contact with delta > 0 in (i, partner) order, each with its force and updated
 * history; per-owner force (gravity first, then contacts) and torque sums.
 * The contacts of each block of spheres are found independently (in parallel when
 * w->n_threads > 1); the reduction onto the owners then runs serially in (i, partner)
 * order, so every sum, and the result, is the same whatever the thread count. */
#define ORC_BLOCK 64

static int evaluate(const orc_world *w, const double *p, double *F, double *T, contact_buf *out)
{
    const orc_hist *h = (const orc_hist *)w->hist;
    int64_t M = w->n_owner, N = w->n_sphere;
    for (int64_t o = 0; o < M; ++o) {
        double m = w->mass[o];
        int act = owner_is_active(w, o);
        F[3 * o + 0] = act ? m * w->g[0] : 0.0;
        F[3 * o + 1] = act ? m * w->g[1] : 0.0;
        F[3 * o + 2] = act ? m * w->g[2] : 0.0;
        T[3 * o + 0] = 0.0; T[3 * o + 1] = 0.0; T[3 * o + 2] = 0.0;
    }
    grid_ent *ge = NULL;
    int64_t ng = 0, *home = NULL, *start = NULL, dims[3] = {0, 0, 0};
    int use_grid = 0;
    /* the grid finds pairs that can touch; a bond also acts across a gap, so the bonded
     * model takes the plain loop */
    if (w->cell_list && w->model == ORC_MODEL_HERTZ_MINDLIN) {
        use_grid = grid_build(w, p, &ge, &ng, &home);
        if (use_grid < 0) return use_grid;
        if (use_grid) start = grid_starts(ge, ng, dims);
    }
    int64_t nblk = (N + ORC_BLOCK - 1) / ORC_BLOCK;
    contact_buf *blk = (contact_buf *)calloc((size_t)(nblk > 0 ? nblk : 1), sizeof(contact_buf));
    if (!blk) { free(start); free(home); free(ge); return ORC_ERR_NOMEM; }
    int err = 0;
    const int nt = n_threads(w);
    (void)nt;
#pragma omp parallel num_threads(nt) if (nt > 1)
    {
        int64_t *cand = use_grid ? (int64_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(int64_t)) : NULL;
        int my_err = (use_grid && !cand) ? ORC_ERR_NOMEM : 0;
#pragma omp for schedule(dynamic, 1)
        for (int64_t b = 0; b < nblk; ++b) {
            int64_t i_end = (b + 1) * ORC_BLOCK < N ? (b + 1) * ORC_BLOCK : N;
            for (int64_t i = b * ORC_BLOCK; i < i_end && !my_err; ++i) {
                if (!owner_is_active(w, w->owner[i])) continue;
                orc_contact rec;
                /* sphere partners j > i first, then walls in ascending id */
                if (use_grid) {
                    int64_t nc = grid_candidates(ge, ng, start, dims, &home[3 * i], i, cand);
                    for (int64_t a = 0; a < nc && !my_err; ++a)
                        if (contact_of(w, p, h, i, cand[a], &rec)) my_err = cbuf_push(&blk[b], &rec);
                    for (int64_t jj = N; jj < N + w->n_wall && !my_err; ++jj)
                        if (contact_of(w, p, h, i, jj, &rec)) my_err = cbuf_push(&blk[b], &rec);
                } else {
                    for (int64_t jj = i + 1; jj < N + w->n_wall && !my_err; ++jj)
                        if (contact_of(w, p, h, i, jj, &rec)) my_err = cbuf_push(&blk[b], &rec);
                }
            }
        }
        free(cand);
        if (my_err) {
#pragma omp critical
            err = my_err;
        }
    }
    for (int64_t b = 0; b < nblk && !err; ++b)
        for (int64_t k = 0; k < blk[b].n && !err; ++k) {
            add_to_owners(w, &blk[b].c[k], F, T);
            if (out) err = cbuf_push(out, &blk[b].c[k]);
        }
    for (int64_t b = 0; b < nblk; ++b) free(blk[b].c);
    free(blk);
    free(start);
    free(home);
    free(ge);
    return err;
}

int orc_eval(const orc_world *w, double *F, double *T, int64_t cap, int64_t *count, orc_contact *contacts)
{
    double *p = (double *)malloc((size_t)(w->n_sphere > 0 ? w->n_sphere : 1) * 3 * sizeof(double));
    if (!p) return ORC_ERR_NOMEM;
    orc_sphere_positions(w, p);
    contact_buf buf = {0, 0, NULL};
    int e = evaluate(w, p, F, T, &buf);
    free(p);
    if (e) { free(buf.c); return e; }
    if (count) *count = buf.n;
    if (contacts) {
        int64_t nc = buf.n < cap ? buf.n : cap;
        memcpy(contacts, buf.c, (size_t)nc * sizeof(orc_contact));
    }
    free(buf.c);
    if (contacts && buf.n > cap) return ORC_ERR_CAPACITY;
    return 0;
}

/* ------------------------------------------------------------------ integration */

/* Semi-implicit Euler (reading adopted for the unstated scheme): v, then wb with the
 * body-frame Euler equations, then x with the new v, then q with the new wb. */
static void integrate_owner(orc_world *w, int64_t o, const double Fo[3], const double To[3])
{
    double h = w->h, m = w->mass[o];
    double *v = &w->v[3 * o], *x = &w->x[3 * o], *wb = &w->wb[3 * o], *q = &w->q[4 * o];
    const double *I = &w->moi[3 * o];
    const orc_family_motion *pm = w->motion ? &w->motion[owner_family(w, o)] : NULL;
    for (int k = 0; k < 3; ++k) {
        double a = Fo[k] / m;
        v[k] = v[k] + h * a;
    }
    if (pm && pm->fix_v) { v[0] = pm->v[0]; v[1] = pm->v[1]; v[2] = pm->v[2]; }
    if (pm && pm->fix_w) {
        /* prescribed angular velocity (global frame): the orientation turns by it */
        for (int k = 0; k < 3; ++k) x[k] = x[k] + h * v[k];
        double wn = norm3(pm->w);
        if (wn >= 1e-30) {
            double half = 0.5 * h * wn;
            double s = sin(half) / wn;
            double dq[4] = {cos(half), s * pm->w[0], s * pm->w[1], s * pm->w[2]};
            double nq[4];
            quat_mul(dq, q, nq);
            double qn = sqrt(((nq[0] * nq[0] + nq[1] * nq[1]) + nq[2] * nq[2]) + nq[3] * nq[3]);
            q[0] = nq[0] / qn; q[1] = nq[1] / qn; q[2] = nq[2] / qn; q[3] = nq[3] / qn;
        }
        double R[9];
        quat_matrix(q, R);
        mat_tvec(R, pm->w, wb);
        return;
    }
    double R[9], Tb[3];
    quat_matrix(q, R);
    mat_tvec(R, To, Tb);
    double Iw[3] = {I[0] * wb[0], I[1] * wb[1], I[2] * wb[2]};
    double gyro[3] = {0.0, 0.0, 0.0};
    if (w->gyroscopic) cross3(wb, Iw, gyro);
    for (int k = 0; k < 3; ++k) {
        double dw = (Tb[k] - gyro[k]) / I[k];
        wb[k] = wb[k] + h * dw;
    }
    for (int k = 0; k < 3; ++k) x[k] = x[k] + h * v[k];
    double wn = norm3(wb);
    if (wn >= 1e-30) {
        double half = 0.5 * h * wn;
        double s = sin(half) / wn;
        double dq[4] = {cos(half), s * wb[0], s * wb[1], s * wb[2]};
        double nq[4];
        quat_mul(q, dq, nq);
        double qn = sqrt(((nq[0] * nq[0] + nq[1] * nq[1]) + nq[2] * nq[2]) + nq[3] * nq[3]);
        q[0] = nq[0] / qn; q[1] = nq[1] / qn; q[2] = nq[2] / qn; q[3] = nq[3] / qn;
    }
}

static int replace_history(orc_world *w, const contact_buf *b)
{
    orc_hist *h = (orc_hist *)w->hist;
    if (!h) return 0;
    if (hist_reserve(h, b->n)) return ORC_ERR_NOMEM;
    for (int64_t k = 0; k < b->n; ++k) {
        h->i[k] = b->c[k].i; h->j[k] = b->c[k].j;
        h->ut[3 * k] = b->c[k].ut[0]; h->ut[3 * k + 1] = b->c[k].ut[1]; h->ut[3 * k + 2] = b->c[k].ut[2];
        h->age[k] = b->c[k].age;
        memcpy(&h->wc[4 * k], b->c[k].wc, 4 * sizeof(double));
    }
    h->n = b->n;
    return 0;
}

int orc_step(orc_world *w, int64_t nsteps)
{
    int64_t M = w->n_owner, N = w->n_sphere;
    double *p = (double *)malloc((size_t)(N > 0 ? N : 1) * 3 * sizeof(double));
    double *F = (double *)malloc((size_t)(M > 0 ? M : 1) * 3 * sizeof(double));
    double *T = (double *)malloc((size_t)(M > 0 ? M : 1) * 3 * sizeof(double));
    contact_buf buf = {0, 0, NULL};
    int err = 0;
    if (!p || !F || !T) { err = ORC_ERR_NOMEM; goto done; }
    for (int64_t s = 0; s < nsteps; ++s) {
        orc_sphere_positions(w, p);
        buf.n = 0;
        err = evaluate(w, p, F, T, &buf);
        if (err) goto done;
        err = replace_history(w, &buf);
        if (err) goto done;
        const int nt = n_threads(w);
        (void)nt;
#pragma omp parallel for num_threads(nt) if (nt > 1) schedule(static)
        for (int64_t o = 0; o < M; ++o)
            if (owner_is_active(w, o)) integrate_owner(w, o, &F[3 * o], &T[3 * o]);
        if (w->has_sink && w->active) {
            for (int64_t o = 0; o < M; ++o) {
                if (!w->active[o]) continue;
                double d[3] = {w->x[3 * o] - w->sink_p[0], w->x[3 * o + 1] - w->sink_p[1], w->x[3 * o + 2] - w->sink_p[2]};
                if (dot3(d, w->sink_n) < 0.0) {
                    w->active[o] = 0;
                    w->v[3 * o] = w->v[3 * o + 1] = w->v[3 * o + 2] = 0.0;
                    w->wb[3 * o] = w->wb[3 * o + 1] = w->wb[3 * o + 2] = 0.0;
                }
            }
        }
        w->step += 1;
        if (w->v_err > 0.0) {
            for (int64_t o = 0; o < M; ++o) {
                double sp = norm3(&w->v[3 * o]);
                if (!(sp <= w->v_err)) { err = ORC_ERR_DIVERGED; goto done; }
            }
        }
    }
done:
    free(p); free(F); free(T); free(buf.c);
    return err;
}

/* ------------------------------------------------------------------ diagnostics */

/* Neumaier's compensated sum: the running sum and the lost low-order parts. */
typedef struct { double s, c; } csum;

static void csum_add(csum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

static double csum_get(const csum *a) { return a->s + a->c; }

int orc_diagnostics(const orc_world *w, double *ke, double *pe, double *elastic, double *mom, double *angmom)
{
    int64_t M = w->n_owner, N = w->n_sphere;
    csum k = {0.0, 0.0}, u = {0.0, 0.0}, el = {0.0, 0.0};
    csum P[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}}, L[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
    for (int64_t o = 0; o < M; ++o) {
        const double *v = &w->v[3 * o], *x = &w->x[3 * o], *wb = &w->wb[3 * o], *I = &w->moi[3 * o];
        double m = w->mass[o];
        csum_add(&k, 0.5 * m * dot3(v, v));
        csum_add(&k, 0.5 * ((I[0] * wb[0] * wb[0] + I[1] * wb[1] * wb[1]) + I[2] * wb[2] * wb[2]));
        csum_add(&u, -(m * dot3(w->g, x)));
        double mv[3] = {m * v[0], m * v[1], m * v[2]};
        double orb[3], R[9], Iw[3] = {I[0] * wb[0], I[1] * wb[1], I[2] * wb[2]}, spin[3];
        cross3(x, mv, orb);
        quat_matrix(&w->q[4 * o], R);
        mat_vec(R, Iw, spin);
        for (int a = 0; a < 3; ++a) {
            csum_add(&P[a], mv[a]);
            csum_add(&L[a], orb[a]);
            csum_add(&L[a], spin[a]);
        }
    }
    double *p = (double *)malloc((size_t)(N > 0 ? N : 1) * 3 * sizeof(double));
    if (!p) return ORC_ERR_NOMEM;
    orc_sphere_positions(w, p);
    for (int64_t i = 0; i < N; ++i) {
        if (!owner_is_active(w, w->owner[i])) continue;
        for (int64_t jj = i + 1; jj < N + w->n_wall; ++jj) {
            contact_in ci;
            if (jj < N) {
                if (w->owner[jj] == w->owner[i] || !owner_is_active(w, w->owner[jj])) continue;
                if (!sphere_pair_contact(w, p, i, jj, &ci)) continue;
            } else {
                if (!sphere_wall_contact(w, p, i, (int32_t)(jj - N), &ci)) continue;
            }
            csum_add(&el, (8.0 / 15.0) * ci.Estar * sqrt(ci.Rbar) * ci.delta * ci.delta * sqrt(ci.delta));
        }
    }
    free(p);
    if (ke) *ke = csum_get(&k);
    if (pe) *pe = csum_get(&u);
    if (elastic) *elastic = csum_get(&el);
    if (mom) { for (int a = 0; a < 3; ++a) mom[a] = csum_get(&P[a]); }
    if (angmom) { for (int a = 0; a < 3; ++a) angmom[a] = csum_get(&L[a]); }
    return 0;
}
