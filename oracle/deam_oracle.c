/*
 * Plain, slow FP64 CPU oracle of MAR-DEAM (dual-energy alternating minimisation
 * with metal-trace substitution), arXiv 2202.00116.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path; the two meet only through the
 * seeded inputs of the `synth` module.
 *
 * Every function below is a direct transcription of a definition:
 *   - system operator h(x, y) (Eq. 8, "system operator of the helical fan-beam
 *     CT system"; discretisation: Joseph's method, bilinear in the two
 *     non-dominant axes, voxel-centre planes, dominant axis x when |u_x| >= |u_y|,
 *     taps outside the volume are zero);
 *   - polyenergetic forward model g_j(y:c) = sum_E I0_j(y,E) exp(-sum_x h sum_i mu_i c_i)
 *     (Eq. 8), with I0_j(y,E) = I0_j(E) * bowtie(channel);
 *   - I-divergence I(d||g) = sum d ln(d/g) - d + g (Eq. 5), restricted to rays with
 *     T(y) < t, where T(y) = sum_x h(x,y) M(x) is the metal trace (Sec. 2.1);
 *   - p-step: on the linear family of Eq. (10) the minimiser is p = q d~/g, and on
 *     metal-trace rays p = q (Eq. 11 and the sentence after it);
 *   - c-step: c_i <- c_i - (1/Z) ln(b^_i / b~_i), with
 *     b~_i(x) = sum_{y,E} h mu_i q and b^_i(x) = sum_{y,E} h mu_i p, and the scalar
 *     Z = max_E (mu_1 + mu_2)(E) * max_y sum_x h(x,y) (active bins only).  The paper
 *     cites this update from O'Sullivan & Benac instead of printing it; it follows
 *     from Eqs. (5), (8)-(11) by the alternating-minimisation surrogate argument.
 *     Voxels with b~_i <= 0 or b^_i <= 0 are left unchanged.
 *   - regularised c-step (Eqs. 6-7): see or_iterate_reg below.
 *
 * Layouts: image [nz][ny][nx][2] (c_1, c_2 interleaved), rays [V][R][K] with the
 * per-ray pair last, measurements d [2][V][R][K] (j = L, H), spectra [2][nE].
 * Metal masks are uint8 [V][R][K] with bit j set when ray y lies on the metal
 * trace T_j of spectrum j (Sec. 2.1: the traces differ when the two spectra's
 * system operators differ; with one operator both bits are set together).
 * All arithmetic is double precision.  OpenMP runs independent rays in parallel;
 * backprojection scatters with atomic adds.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#include "or_types.h"

int or_max_taps(const or_geometry *g) { return 4 * (g->nx > g->ny ? g->nx : g->ny); }

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Source point s and (unnormalised) ray vector u of ray (v, r, k). */
static void ray_of(const or_geometry *g, long v, int r, int k, double s[3], double u[3]) {
    double beta = g->start_angle + 2.0 * M_PI * (double)v / g->views_per_rotation;
    double gam = (k - (g->n_channels - 1) / 2.0 + g->channel_offset) * g->channel_pitch;
    double w = (r - (g->n_rows - 1) / 2.0 + g->row_offset) * g->row_pitch;
    s[0] = g->sid * cos(beta);
    s[1] = g->sid * sin(beta);
    s[2] = g->z_start + g->feed * (double)v / g->views_per_rotation;
    u[0] = -g->sdd * cos(beta + gam);
    u[1] = -g->sdd * sin(beta + gam);
    u[2] = w;
}

/* All nonzero h(x, y) of one ray (Joseph's method). Returns the tap count. */
int or_ray_taps(const or_geometry *g, long v, int r, int k, or_tap *T) {
    double s[3], u[3];
    ray_of(g, v, r, k, s, u);
    const double X0 = g->cx - (g->nx - 1) / 2.0 * g->dx;
    const double Y0 = g->cy - (g->ny - 1) / 2.0 * g->dy;
    const double Z0 = g->cz - (g->nz - 1) / 2.0 * g->dz;
    const double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    int n = 0;
    if (fabs(u[0]) >= fabs(u[1])) {
        /* x-dominant: one sample per plane x = X(ix) */
        const double L = g->dx * un / fabs(u[0]);
        for (int ix = 0; ix < g->nx; ix++) {
            double t = (X0 + ix * g->dx - s[0]) / u[0];
            double fy = (s[1] + t * u[1] - Y0) / g->dy;
            double fz = (s[2] + t * u[2] - Z0) / g->dz;
            if (!(fy > -2.0 && fy < g->ny + 1.0 && fz > -2.0 && fz < g->nz + 1.0)) continue;
            double jf = floor(fy), mf = floor(fz);
            double a = fy - jf, b = fz - mf;
            int j = (int)jf, m = (int)mf;
            for (int dm = 0; dm < 2; dm++) {
                int iz = m + dm;
                if (iz < 0 || iz >= g->nz) continue;
                double wz = dm ? b : 1.0 - b;
                for (int dj = 0; dj < 2; dj++) {
                    int iy = j + dj;
                    if (iy < 0 || iy >= g->ny) continue;
                    double w = L * (dj ? a : 1.0 - a) * wz;
                    if (w == 0.0) continue;
                    T[n].idx = ((long)iz * g->ny + iy) * g->nx + ix;
                    T[n].w = w;
                    n++;
                }
            }
        }
    } else {
        /* y-dominant: one sample per plane y = Y(iy) */
        const double L = g->dy * un / fabs(u[1]);
        for (int iy = 0; iy < g->ny; iy++) {
            double t = (Y0 + iy * g->dy - s[1]) / u[1];
            double fx = (s[0] + t * u[0] - X0) / g->dx;
            double fz = (s[2] + t * u[2] - Z0) / g->dz;
            if (!(fx > -2.0 && fx < g->nx + 1.0 && fz > -2.0 && fz < g->nz + 1.0)) continue;
            double jf = floor(fx), mf = floor(fz);
            double a = fx - jf, b = fz - mf;
            int j = (int)jf, m = (int)mf;
            for (int dm = 0; dm < 2; dm++) {
                int iz = m + dm;
                if (iz < 0 || iz >= g->nz) continue;
                double wz = dm ? b : 1.0 - b;
                for (int dj = 0; dj < 2; dj++) {
                    int ix = j + dj;
                    if (ix < 0 || ix >= g->nx) continue;
                    double w = L * (dj ? a : 1.0 - a) * wz;
                    if (w == 0.0) continue;
                    T[n].idx = ((long)iz * g->ny + iy) * g->nx + ix;
                    T[n].w = w;
                    n++;
                }
            }
        }
    }
    return n;
}

static long n_rays_in(const or_geometry *g, int v0, int v1) {
    return (long)(v1 - v0) * g->n_rows * g->n_channels;
}

/* Forward projection l_i(y) = sum_x h(x,y) c_i(x) for views [v0, v1).
 * c: [nz][ny][nx][2]; l: [V][R][K][2] (only the selected views are written). */
void or_forward(const or_geometry *g, const double *c, double *l, int v0, int v1) {
    const int RK = g->n_rows * g->n_channels;
    const long n = n_rays_in(g, v0, v1);
#pragma omp parallel
    {
        or_tap *T = (or_tap *)malloc(sizeof(or_tap) * or_max_taps(g));
#pragma omp for schedule(dynamic, 64)
        for (long q = 0; q < n; q++) {
            long v = v0 + q / RK;
            int r = (int)((q % RK) / g->n_channels), k = (int)(q % g->n_channels);
            int nt = or_ray_taps(g, v, r, k, T);
            double a1 = 0.0, a2 = 0.0;
            for (int t = 0; t < nt; t++) {
                a1 += T[t].w * c[2 * T[t].idx];
                a2 += T[t].w * c[2 * T[t].idx + 1];
            }
            long y = v * RK + (long)r * g->n_channels + k;
            l[2 * y] = a1;
            l[2 * y + 1] = a2;
        }
        free(T);
    }
}

/* Forward projection of selected rays (ray index = (v*R + r)*K + k). */
void or_forward_rays(const or_geometry *g, const double *c, const int64_t *rays, long n, double *out) {
    const int RK = g->n_rows * g->n_channels;
#pragma omp parallel
    {
        or_tap *T = (or_tap *)malloc(sizeof(or_tap) * or_max_taps(g));
#pragma omp for schedule(dynamic, 16)
        for (long q = 0; q < n; q++) {
            long y = rays[q];
            long v = y / RK;
            int r = (int)((y % RK) / g->n_channels), k = (int)(y % g->n_channels);
            int nt = or_ray_taps(g, v, r, k, T);
            double a1 = 0.0, a2 = 0.0;
            for (int t = 0; t < nt; t++) {
                a1 += T[t].w * c[2 * T[t].idx];
                a2 += T[t].w * c[2 * T[t].idx + 1];
            }
            out[2 * q] = a1;
            out[2 * q + 1] = a2;
        }
        free(T);
    }
}

/* Adjoint (backprojection) img_i(x) = sum_{y in views [v0,v1)} h(x,y) y_i(y).
 * img is overwritten. */
void or_adjoint(const or_geometry *g, const double *yv, double *img, int v0, int v1) {
    const int RK = g->n_rows * g->n_channels;
    const long nvox = (long)g->nx * g->ny * g->nz;
    const long n = n_rays_in(g, v0, v1);
    memset(img, 0, sizeof(double) * 2 * nvox);
#pragma omp parallel
    {
        or_tap *T = (or_tap *)malloc(sizeof(or_tap) * or_max_taps(g));
#pragma omp for schedule(dynamic, 64)
        for (long q = 0; q < n; q++) {
            long v = v0 + q / RK;
            int r = (int)((q % RK) / g->n_channels), k = (int)(q % g->n_channels);
            long y = v * RK + (long)r * g->n_channels + k;
            double b1 = yv[2 * y], b2 = yv[2 * y + 1];
            if (b1 == 0.0 && b2 == 0.0) continue;
            int nt = or_ray_taps(g, v, r, k, T);
            for (int t = 0; t < nt; t++) {
#pragma omp atomic
                img[2 * T[t].idx] += T[t].w * b1;
#pragma omp atomic
                img[2 * T[t].idx + 1] += T[t].w * b2;
            }
        }
        free(T);
    }
}

/* Eq. (8) for one ray and one spectrum j, with the two spectral moments the
 * c-step needs: g = sum_E q, S_i = sum_E mu_i(E) q, q = I0_j(E) b(k) exp(-mu.l). */
static void spectral_sums(const or_model *m, int j, int k, double l1, double l2,
                          double *g, double *S1, double *S2) {
    double b = m->bowtie ? m->bowtie[k] : 1.0;
    double gg = 0.0, s1 = 0.0, s2 = 0.0;
    for (int e = 0; e < m->n_e; e++) {
        double I0 = m->I0[j * m->n_e + e] * b;
        if (I0 == 0.0) continue;
        double mu1 = m->mu[e], mu2 = m->mu[m->n_e + e];
        double q = I0 * exp(-(mu1 * l1 + mu2 * l2));
        gg += q;
        s1 += mu1 * q;
        s2 += mu2 * q;
    }
    *g = gg;
    *S1 = s1;
    *S2 = s2;
}

/* Expected counts g_j(y) (Eq. 8) for all rays of views [v0, v1) from line
 * integrals l [V][R][K][2]; g is [2][V][R][K]. */
void or_expected(const or_geometry *g, const or_model *m, const double *l, double *gout, int v0, int v1) {
    const int RK = g->n_rows * g->n_channels;
    const long nrays = (long)g->n_views * RK;
    const long n = n_rays_in(g, v0, v1);
#pragma omp parallel for schedule(static)
    for (long q = 0; q < n; q++) {
        long y = (long)v0 * RK + q;
        int k = (int)(y % g->n_channels);
        for (int j = 0; j < 2; j++) {
            double gg, s1, s2;
            spectral_sums(m, j, k, l[2 * y], l[2 * y + 1], &gg, &s1, &s2);
            gout[j * nrays + y] = gg;
        }
    }
}

/* One I-divergence term d ln(d/g) - d + g (Eq. 5), with 0 ln 0 = 0. */
static double idiv_term(double d, double g) {
    if (d > 0.0) return d * log(d / g) - d + g;
    return g;
}

/* Per-ray quantities of one DEAM iteration for the listed rays:
 * l [n][2], g [n][2] (j = L, H), payload [n][4] = (B~_1, B~_2, B^_1, B^_2) where
 * B~_i = sum_j S_ij and B^_i = sum_j r_j S_ij, r_j = 1 on metal rays and d~_j/g_j
 * elsewhere, and the objective contribution f [n] (0 on metal rays).
 * d is [2][V][R][K], mask [V][R][K] (nonzero = metal trace). */
void or_ray_model(const or_geometry *g, const or_model *m, const double *c, const double *d,
                  const uint8_t *mask, const int64_t *rays, long n,
                  double *l, double *gout, double *payload, double *f) {
    const int RK = g->n_rows * g->n_channels;
    const long nrays = (long)g->n_views * RK;
#pragma omp parallel
    {
        or_tap *T = (or_tap *)malloc(sizeof(or_tap) * or_max_taps(g));
#pragma omp for schedule(dynamic, 16)
        for (long q = 0; q < n; q++) {
            long y = rays[q];
            long v = y / RK;
            int r = (int)((y % RK) / g->n_channels), k = (int)(y % g->n_channels);
            int nt = or_ray_taps(g, v, r, k, T);
            double l1 = 0.0, l2 = 0.0;
            for (int t = 0; t < nt; t++) {
                l1 += T[t].w * c[2 * T[t].idx];
                l2 += T[t].w * c[2 * T[t].idx + 1];
            }
            double Bt1 = 0.0, Bt2 = 0.0, Bh1 = 0.0, Bh2 = 0.0, ff = 0.0;
            for (int j = 0; j < 2; j++) {
                double gg, s1, s2;
                spectral_sums(m, j, k, l1, l2, &gg, &s1, &s2);
                double dt = d[j * nrays + y] > 0.0 ? d[j * nrays + y] : 0.0;
                double rj = 1.0;   /* where g = 0 every q is 0 and r*S = 0 for any r */
                if (!(mask[y] & (1u << j))) {   /* bit j: ray on the metal trace T_j of spectrum j */
                    if (gg > 0.0) rj = dt / gg;
                    ff += idiv_term(dt, gg);
                }
                Bt1 += s1;
                Bt2 += s2;
                Bh1 += rj * s1;
                Bh2 += rj * s2;
                gout[2 * q + j] = gg;
            }
            l[2 * q] = l1;
            l[2 * q + 1] = l2;
            payload[4 * q + 0] = Bt1;
            payload[4 * q + 1] = Bt2;
            payload[4 * q + 2] = Bh1;
            payload[4 * q + 3] = Bh2;
            f[q] = ff;
        }
        free(T);
    }
}

/* One pass over the rays of views [v0, v1): objective F and the backprojected
 * sums bt = b~ and bh = b^ ([nvox][2] each, overwritten). Returns F. */
static double ray_pass(const or_geometry *g, const or_model *m, const double *c, const double *d,
                       const uint8_t *mask, double *bt, double *bh, int v0, int v1) {
    const int RK = g->n_rows * g->n_channels;
    const long nrays = (long)g->n_views * RK;
    const long nvox = (long)g->nx * g->ny * g->nz;
    const long n = n_rays_in(g, v0, v1);
    double F = 0.0;
    if (bt) memset(bt, 0, sizeof(double) * 2 * nvox);
    if (bh) memset(bh, 0, sizeof(double) * 2 * nvox);
#pragma omp parallel reduction(+ : F)
    {
        or_tap *T = (or_tap *)malloc(sizeof(or_tap) * or_max_taps(g));
#pragma omp for schedule(dynamic, 64)
        for (long q = 0; q < n; q++) {
            long v = v0 + q / RK;
            int r = (int)((q % RK) / g->n_channels), k = (int)(q % g->n_channels);
            long y = v * RK + (long)r * g->n_channels + k;
            int nt = or_ray_taps(g, v, r, k, T);
            double l1 = 0.0, l2 = 0.0;
            for (int t = 0; t < nt; t++) {
                l1 += T[t].w * c[2 * T[t].idx];
                l2 += T[t].w * c[2 * T[t].idx + 1];
            }
            double Bt1 = 0.0, Bt2 = 0.0, Bh1 = 0.0, Bh2 = 0.0;
            for (int j = 0; j < 2; j++) {
                double gg, s1, s2;
                spectral_sums(m, j, k, l1, l2, &gg, &s1, &s2);
                double dt = d[j * nrays + y] > 0.0 ? d[j * nrays + y] : 0.0;
                double rj = 1.0;   /* where g = 0 every q is 0 and r*S = 0 for any r */
                if (!(mask[y] & (1u << j))) {   /* bit j: ray on the metal trace T_j of spectrum j */
                    if (gg > 0.0) rj = dt / gg;
                    F += idiv_term(dt, gg);
                }
                Bt1 += s1;
                Bt2 += s2;
                Bh1 += rj * s1;
                Bh2 += rj * s2;
            }
            if (!bt) continue;
            for (int t = 0; t < nt; t++) {
                long x = T[t].idx;
                double w = T[t].w;
#pragma omp atomic
                bt[2 * x] += w * Bt1;
#pragma omp atomic
                bt[2 * x + 1] += w * Bt2;
#pragma omp atomic
                bh[2 * x] += w * Bh1;
#pragma omp atomic
                bh[2 * x + 1] += w * Bh2;
            }
        }
        free(T);
    }
    return F;
}

/* The objective F(c) = sum_j sum_{y: T(y) < t} I(d~_j(y) || g_j(y:c)) (Eq. 5 with
 * the substitution of Eqs. 2-3: metal-trace rays contribute nothing). */
double or_objective(const or_geometry *g, const or_model *m, const double *c, const double *d,
                    const uint8_t *mask) {
    return ray_pass(g, m, c, d, mask, NULL, NULL, 0, g->n_views);
}

/* Backprojected spectral sums b~ and b^ (both [nz][ny][nx][2]) and F(c). */
double or_backprojected_sums(const or_geometry *g, const or_model *m, const double *c, const double *d,
                             const uint8_t *mask, double *bt, double *bh, int v0, int v1) {
    return ray_pass(g, m, c, d, mask, bt, bh, v0, v1);
}

/* Normaliser Z = max over active bins of (mu_1 + mu_2)(E) times max_y sum_x h(x,y). */
double or_normaliser(const or_geometry *g, const or_model *m) {
    const int RK = g->n_rows * g->n_channels;
    const long n = (long)g->n_views * RK;
    double hmax = 0.0;
#pragma omp parallel reduction(max : hmax)
    {
        or_tap *T = (or_tap *)malloc(sizeof(or_tap) * or_max_taps(g));
#pragma omp for schedule(dynamic, 64)
        for (long q = 0; q < n; q++) {
            long v = q / RK;
            int r = (int)((q % RK) / g->n_channels), k = (int)(q % g->n_channels);
            int nt = or_ray_taps(g, v, r, k, T);
            double s = 0.0;
            for (int t = 0; t < nt; t++) s += T[t].w;
            if (s > hmax) hmax = s;
        }
        free(T);
    }
    double mumax = 0.0;
    for (int e = 0; e < m->n_e; e++) {
        if (m->I0[e] == 0.0 && m->I0[m->n_e + e] == 0.0) continue;
        double s = m->mu[e] + m->mu[m->n_e + e];
        if (s > mumax) mumax = s;
    }
    return mumax * hmax;
}

/* Metal trace T(y) = sum_x h(x,y) M(x) (Sec. 2.1) and mask = (T >= t) for both
 * spectra (bits 0 and 1: one system operator). */
void or_metal_trace(const or_geometry *g, const double *M, double t, double *T_out, uint8_t *mask) {
    const int RK = g->n_rows * g->n_channels;
    const long n = (long)g->n_views * RK;
#pragma omp parallel
    {
        or_tap *T = (or_tap *)malloc(sizeof(or_tap) * or_max_taps(g));
#pragma omp for schedule(dynamic, 64)
        for (long q = 0; q < n; q++) {
            long v = q / RK;
            int r = (int)((q % RK) / g->n_channels), k = (int)(q % g->n_channels);
            int nt = or_ray_taps(g, v, r, k, T);
            double s = 0.0;
            for (int i = 0; i < nt; i++) s += T[i].w * M[T[i].idx];
            T_out[q] = s;
            mask[q] = (uint8_t)(s >= t ? 3 : 0);
        }
        free(T);
    }
}

/* ---- Penalty of Eqs. (6)-(7) ------------------------------------------------
 * R(c) = lambda sum_i sum_x sum_{x~ in N_x} w(x,x~) phi(c_i(x) - c_i(x~)),
 * N_x = the 26 neighbours of x inside the volume, w = 1 / physical distance,
 * phi(u) = delta^2 (|u|/delta - log(1 + |u|/delta)) (the printed phi has
 * "log(1 - |t/delta|)", undefined for |t| >= delta and not convex; this is the
 * convex reading), so phi'(u) = u / (1 + |u|/delta), phi''(u) = 1/(1 + |u|/delta)^2. */
double or_phi(double u, double delta) {
    double a = fabs(u) / delta;
    return delta * delta * (a - log1p(a));
}

static double phi_d1(double u, double delta) { return u / (1.0 + fabs(u) / delta); }

static double phi_d2(double u, double delta) {
    double a = 1.0 + fabs(u) / delta;
    return 1.0 / (a * a);
}

static double nb_weight(const or_geometry *g, int ox, int oy, int oz) {
    double x = ox * g->dx, y = oy * g->dy, z = oz * g->dz;
    return 1.0 / sqrt(x * x + y * y + z * z);
}

/* R(c) over the whole volume (each ordered pair (x, x~) counted, as printed). */
double or_penalty(const or_geometry *g, const double *c, double lambda, double delta) {
    double R = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : R) collapse(2)
    for (int iz = 0; iz < g->nz; iz++)
        for (int iy = 0; iy < g->ny; iy++)
            for (int ix = 0; ix < g->nx; ix++) {
                long x = ((long)iz * g->ny + iy) * g->nx + ix;
                for (int oz = -1; oz <= 1; oz++)
                    for (int oy = -1; oy <= 1; oy++)
                        for (int ox = -1; ox <= 1; ox++) {
                            if (!ox && !oy && !oz) continue;
                            int jx = ix + ox, jy = iy + oy, jz = iz + oz;
                            if (jx < 0 || jy < 0 || jz < 0 || jx >= g->nx || jy >= g->ny || jz >= g->nz) continue;
                            long xn = ((long)jz * g->ny + jy) * g->nx + jx;
                            double w = nb_weight(g, ox, oy, oz);
                            for (int i = 0; i < 2; i++) R += w * or_phi(c[2 * x + i] - c[2 * xn + i], delta);
                        }
            }
    return lambda * R;
}

/* Regularised c-step (De Pierro's separable surrogate of the convex pairwise
 * penalty added to the DEAM surrogate).  Summing the two halves of every pair
 * that involves x, voxel x and component i minimise, over t = c_i(x),
 *   G(t) = bh (t - ck) + (bt / Z) exp(-Z (t - ck)) + lambda sum_x~ w phi(2 t - ck - ck_x~)
 * whose derivative is increasing.  Root of G' by bisection-safeguarded Newton
 * in a bracket that holds because |phi'| < delta. */
static double reg_solve(double ck, double bt, double bh, double Z, double lambda, double delta, const double *m,
                        const double *w, int nn) {
    /* m[n] = ck + ck_x~; G'(t) = bh - bt e^{-Z(t-ck)} + 2 lambda sum w phi'(2t - m) */
    double pmax = 0.0, lo, hi;
    for (int n = 0; n < nn; n++) pmax += 2.0 * lambda * w[n] * delta;
    if (bt > 0.0) {
        double a = bh + pmax, b = bh - pmax;
        lo = ck - log(a / bt) / Z;
        hi = b > 0.0 ? ck - log(b / bt) / Z : 1e300;
        if (!(hi < 1e300)) {
            /* G' < 0 only below some finite t: widen until G'(hi) > 0 */
            hi = lo + 1.0;
            for (int it = 0; it < 200; it++) {
                double gp = bh - bt * exp(-Z * (hi - ck));
                for (int n = 0; n < nn; n++) gp += 2.0 * lambda * w[n] * phi_d1(2.0 * hi - m[n], delta);
                if (gp > 0.0) break;
                hi = lo + 2.0 * (hi - lo);
            }
        }
    } else {
        lo = 1e300;
        hi = -1e300;
        for (int n = 0; n < nn; n++) {
            lo = fmin(lo, 0.5 * m[n]);
            hi = fmax(hi, 0.5 * m[n]);
        }
    }
    double t = 0.5 * (lo + hi);
    for (int it = 0; it < 200; it++) {
        double gp = bh, gpp = 0.0;
        if (bt > 0.0) {
            double e = bt * exp(-Z * (t - ck));
            gp -= e;
            gpp += Z * e;
        }
        for (int n = 0; n < nn; n++) {
            double u = 2.0 * t - m[n];
            gp += 2.0 * lambda * w[n] * phi_d1(u, delta);
            gpp += 4.0 * lambda * w[n] * phi_d2(u, delta);
        }
        if (gp > 0.0) hi = t;
        else lo = t;
        double tn = gpp > 0.0 ? t - gp / gpp : 0.5 * (lo + hi);
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        if (fabs(tn - t) <= 1e-15 * (1.0 + fabs(t)) || hi - lo <= 1e-15 * (1.0 + fabs(t))) {
            t = tn;
            break;
        }
        t = tn;
    }
    return t;
}

static long c_step_reg(const or_geometry *g, double *c, const double *bt, const double *bh, double Z, double lambda,
                       double delta, int clamp_nonneg) {
    const long nvox = (long)g->nx * g->ny * g->nz;
    double *ck = (double *)malloc(sizeof(double) * 2 * nvox);
    memcpy(ck, c, sizeof(double) * 2 * nvox);
    long skipped = 0;
#pragma omp parallel for schedule(static) reduction(+ : skipped) collapse(2)
    for (int iz = 0; iz < g->nz; iz++)
        for (int iy = 0; iy < g->ny; iy++)
            for (int ix = 0; ix < g->nx; ix++) {
                long x = ((long)iz * g->ny + iy) * g->nx + ix;
                for (int i = 0; i < 2; i++) {
                    double m[26], w[26];
                    int nn = 0;
                    for (int oz = -1; oz <= 1; oz++)
                        for (int oy = -1; oy <= 1; oy++)
                            for (int ox = -1; ox <= 1; ox++) {
                                if (!ox && !oy && !oz) continue;
                                int jx = ix + ox, jy = iy + oy, jz = iz + oz;
                                if (jx < 0 || jy < 0 || jz < 0 || jx >= g->nx || jy >= g->ny || jz >= g->nz) continue;
                                long xn = ((long)jz * g->ny + jy) * g->nx + jx;
                                m[nn] = ck[2 * x + i] + ck[2 * xn + i];
                                w[nn] = nb_weight(g, ox, oy, oz);
                                nn++;
                            }
                    double b_t = bt[2 * x + i], b_h = bh[2 * x + i];
                    if (b_t > 0.0 && !(b_h > 0.0)) {  /* b^ <= 0: the data term is unbounded below */
                        skipped++;
                        continue;
                    }
                    if (!(b_t > 0.0) && nn == 0) {
                        skipped++;
                        continue;
                    }
                    double t = reg_solve(ck[2 * x + i], b_t > 0.0 ? b_t : 0.0, b_t > 0.0 ? b_h : 0.0, Z, lambda,
                                         delta, m, w, nn);
                    if (clamp_nonneg && t < 0.0) t = 0.0;
                    c[2 * x + i] = t;
                }
            }
    free(ck);
    return skipped;
}

/* The c-step: c_i <- c_i - ln(b^_i / b~_i) / Z where both sums are positive.
 * Returns the number of (voxel, component) pairs left unchanged. */
static long c_step(long nvox, double *c, const double *bt, const double *bh, double Z, int clamp_nonneg) {
    long skipped = 0;
#pragma omp parallel for schedule(static) reduction(+ : skipped)
    for (long x = 0; x < 2 * nvox; x++) {
        if (bt[x] > 0.0 && bh[x] > 0.0) {
            c[x] -= log(bh[x] / bt[x]) / Z;
            if (clamp_nonneg && c[x] < 0.0) c[x] = 0.0;
        } else {
            skipped++;
        }
    }
    return skipped;
}

/* n_iter MAR-DEAM iterations in place on c.  hist[k] = F(c^k) before update k.
 * Z <= 0 selects the normaliser above.  Returns the skip count of the last c-step.
 * Views [v0, v1) restrict the rays used (the full method uses all views). */
long or_iterate_reg(const or_geometry *g, const or_model *m, double *c, const double *d, const uint8_t *mask,
                    int n_iter, double *hist, double *hist_R, double Z, int clamp_nonneg, double lambda,
                    double delta) {
    const long nvox = (long)g->nx * g->ny * g->nz;
    if (Z <= 0.0) Z = or_normaliser(g, m);
    double *bt = (double *)malloc(sizeof(double) * 2 * nvox);
    double *bh = (double *)malloc(sizeof(double) * 2 * nvox);
    long skipped = 0;
    for (int it = 0; it < n_iter; it++) {
        double F = ray_pass(g, m, c, d, mask, bt, bh, 0, g->n_views);
        if (hist) hist[it] = F;
        if (hist_R) hist_R[it] = or_penalty(g, c, lambda, delta);
        skipped = c_step_reg(g, c, bt, bh, Z, lambda, delta, clamp_nonneg);
    }
    free(bt);
    free(bh);
    return skipped;
}

long or_iterate(const or_geometry *g, const or_model *m, double *c, const double *d, const uint8_t *mask,
                int n_iter, double *hist, double Z, int clamp_nonneg, int v0, int v1) {
    const long nvox = (long)g->nx * g->ny * g->nz;
    if (Z <= 0.0) Z = or_normaliser(g, m);
    double *bt = (double *)malloc(sizeof(double) * 2 * nvox);
    double *bh = (double *)malloc(sizeof(double) * 2 * nvox);
    long skipped = 0;
    for (int it = 0; it < n_iter; it++) {
        double F = ray_pass(g, m, c, d, mask, bt, bh, v0, v1);
        if (hist) hist[it] = F;
        skipped = c_step(nvox, c, bt, bh, Z, clamp_nonneg);
    }
    free(bt);
    free(bh);
    return skipped;
}

/* Gradient of F with respect to c: dF/dc_i(x) = b^_i(x) - b~_i(x) (differentiate
 * Eq. 5 through Eq. 8).  grad is [nz][ny][nx][2]. */
void or_gradient(const or_geometry *g, const or_model *m, const double *c, const double *d,
                 const uint8_t *mask, double *grad) {
    const long nvox = (long)g->nx * g->ny * g->nz;
    double *bt = (double *)malloc(sizeof(double) * 2 * nvox);
    double *bh = (double *)malloc(sizeof(double) * 2 * nvox);
    ray_pass(g, m, c, d, mask, bt, bh, 0, g->n_views);
    for (long x = 0; x < 2 * nvox; x++) grad[x] = bh[x] - bt[x];
    free(bt);
    free(bh);
}
