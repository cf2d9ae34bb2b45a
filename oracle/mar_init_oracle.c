/*
 * FP64 oracle of the MAR initialisation (Sec. 2.2 of arXiv 2202.00116):
 * the measured sinograms of both spectra are completed across the metal trace
 * by normalised metal-artifact reduction (NMAR: the sinogram is divided by the
 * forward projection of a prior image, interpolated linearly across the trace,
 * and multiplied back), reconstructed by filtered backprojection, and split
 * into the two basis components by the image-domain decomposition of Eq. (4)
 * with calibrated weights.  The prior image thresholds a single-energy FBP
 * image (air / soft tissue / kept bone values).
 *
 * TEST INFRASTRUCTURE ONLY (same rules as deam_oracle.c).
 *
 * Readings where the paper is silent (each is a parameter or a stated choice):
 *  - sinogram p_j(y) = ln(I0_j(y) / max(d_j(y), floor)), I0_j(y) = sum_E I0_j(E) b(k);
 *  - the prior comes from the FBP of the chosen spectrum's sinogram with the trace
 *    completed by plain linear interpolation (prior == 1), filtered by n passes
 *    of an in-plane [1,2,1]/4 smoothing in x and y, and thresholded into
 *    0 (f < t_air), a soft-tissue value (t_air <= f < t_bone) and f (f >= t_bone);
 *  - NMAR normalises by max(prior projection, eps) and interpolates linearly along
 *    the channels of each (view, row) between the nearest rays off the trace of
 *    that spectrum (constant beyond the row ends); rays off the trace keep p;
 *  - FBP: equiangular fan-beam filtered backprojection on the curved detector
 *    (Kak & Slaney, Principles of Computerized Tomographic Imaging, Sec. 3.4.2:
 *    pre-weight D cos(gamma), discrete kernel g(0) = 1/(8 a^2), g(n even) = 0,
 *    g(n odd) = -1/(2 pi^2 sin^2(n a)), a = channel pitch; backprojection weight
 *    1/L^2 with L the source-voxel distance in the plane), extended to the helix
 *    FDK-style: cone pre-weight SDD / sqrt(SDD^2 + w^2), each voxel backprojects
 *    the one rotation of views centred on the view whose source z equals the
 *    voxel's z, rows interpolated linearly at w = (z - z_s) SDD / L and clamped
 *    to the detector's end rows, channels outside the detector contribute 0;
 *  - Eq. (4) with constant calibrated weights mu~_ij (one 2x2 matrix per scan).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#include "or_types.h"

typedef struct {
    double calib[4];  /* mu~_1L, mu~_2L, mu~_1H, mu~_2H of Eq. (4) */
    double t_air, t_bone, soft_value;
    double count_floor, eps;
    int prior_spectrum; /* 0: L, 1: H */
    int prior_smooth;   /* passes of the in-plane [1,2,1]/4 x [1,2,1]/4 filter before thresholding */
} or_mar_params;

/* Line-integral sinograms of both spectra: p [2][V][R][K]. */
void or_log_sinogram(const or_geometry *g, const or_model *m, const double *d, double floor_counts, double *p) {
    const long RK = (long)g->n_rows * g->n_channels, nrays = (long)g->n_views * RK;
    for (int j = 0; j < 2; j++) {
        double tot = 0.0;
        for (int e = 0; e < m->n_e; e++) tot += m->I0[j * m->n_e + e];
#pragma omp parallel for schedule(static)
        for (long y = 0; y < nrays; y++) {
            int k = (int)(y % g->n_channels);
            double I0 = tot * (m->bowtie ? m->bowtie[k] : 1.0);
            double dd = d[j * nrays + y];
            if (dd < floor_counts) dd = floor_counts;
            p[j * nrays + y] = log(I0 / dd);
        }
    }
}

/* Trace completion of one sinogram p [V][R][K] into out: rays with `bit` set in
 * mask are replaced.  With prior (its projection [V][R][K]) the row p/max(prior,
 * eps) is interpolated and multiplied back by max(prior, eps) (NMAR); without,
 * p itself is interpolated (linear interpolation, LI). */
void or_complete_trace(const or_geometry *g, const double *p, const double *prior, const uint8_t *mask, int bit,
                       double eps, double *out) {
    const int K = g->n_channels;
    const long nrows = (long)g->n_views * g->n_rows;
#pragma omp parallel for schedule(static)
    for (long row = 0; row < nrows; row++) {
        const double *pr = p + row * K;
        const double *qr = prior ? prior + row * K : NULL;
        const uint8_t *mr = mask + row * K;
        double *o = out + row * K;
        for (int k = 0; k < K; k++) {
            if (!(mr[k] & (1u << bit))) {
                o[k] = pr[k];
                continue;
            }
            int kl = k - 1, kr = k + 1;
            while (kl >= 0 && (mr[kl] & (1u << bit))) kl--;
            while (kr < K && (mr[kr] & (1u << bit))) kr++;
            double nl = 0.0, nr = 0.0, val;
            if (kl >= 0) nl = qr ? pr[kl] / fmax(qr[kl], eps) : pr[kl];
            if (kr < K) nr = qr ? pr[kr] / fmax(qr[kr], eps) : pr[kr];
            if (kl >= 0 && kr < K)
                val = nl + (nr - nl) * (double)(k - kl) / (double)(kr - kl);
            else if (kl >= 0)
                val = nl;
            else if (kr < K)
                val = nr;
            else
                val = qr ? pr[k] / fmax(qr[k], eps) : pr[k]; /* whole row on the trace: unchanged */
            o[k] = qr ? val * fmax(qr[k], eps) : val;
        }
    }
}

/* Filtered sinogram q [V][R][K] of p [V][R][K]: fan pre-weight SID cos(gamma),
 * cone pre-weight SDD / sqrt(SDD^2 + w^2), equiangular kernel, times a. */
void or_ramp_filter(const or_geometry *g, const double *p, double *q) {
    const int K = g->n_channels, R = g->n_rows;
    const double a = g->channel_pitch;
    double *ker = (double *)malloc(sizeof(double) * (2 * K - 1));
    for (int n = -(K - 1); n <= K - 1; n++) {
        double v;
        if (n == 0)
            v = 1.0 / (8.0 * a * a);
        else if (n % 2 == 0)
            v = 0.0;
        else {
            double s = sin(n * a);
            v = -1.0 / (2.0 * M_PI * M_PI * s * s);
        }
        ker[n + K - 1] = v;
    }
    const long nrows = (long)g->n_views * R;
#pragma omp parallel
    {
        double *pw = (double *)malloc(sizeof(double) * K);
#pragma omp for schedule(static)
        for (long row = 0; row < nrows; row++) {
            int r = (int)(row % R);
            double w = (r - (R - 1) / 2.0 + g->row_offset) * g->row_pitch;
            double cone = g->sdd / sqrt(g->sdd * g->sdd + w * w);
            for (int k = 0; k < K; k++) {
                double gam = (k - (K - 1) / 2.0 + g->channel_offset) * a;
                pw[k] = p[row * K + k] * g->sid * cos(gam) * cone;
            }
            for (int n = 0; n < K; n++) {
                double s = 0.0;
                for (int k = 0; k < K; k++) s += pw[k] * ker[n - k + K - 1];
                q[row * K + n] = a * s;
            }
        }
        free(pw);
    }
    free(ker);
}

/* Views backprojected into a voxel at height Z: [*v0, *v1). */
static void view_window(const or_geometry *g, double Z, long *v0, long *v1) {
    const long N = g->views_per_rotation, V = g->n_views;
    long a = 0, b = V < N ? V : N;
    if (g->feed != 0.0 && g->n_rows > 1) {
        double vc = (Z - g->z_start) * (double)N / g->feed;
        a = (long)ceil(vc - N / 2.0);
        b = a + N;
    }
    if (a < 0) a = 0;
    if (b > V) b = V;
    *v0 = a;
    *v1 = b;
}

/* FBP backprojection value at one voxel (index iz*ny*nx + iy*nx + ix). */
static double fbp_voxel(const or_geometry *g, const double *q, long vi) {
    const int K = g->n_channels, R = g->n_rows;
    const long N = g->views_per_rotation;
    const double X0 = g->cx - (g->nx - 1) / 2.0 * g->dx;
    const double Y0 = g->cy - (g->ny - 1) / 2.0 * g->dy;
    const double Z0 = g->cz - (g->nz - 1) / 2.0 * g->dz;
    const double dbeta = 2.0 * M_PI / (double)N;
    int ix = (int)(vi % g->nx), iy = (int)((vi / g->nx) % g->ny), iz = (int)(vi / ((long)g->nx * g->ny));
    double X = X0 + ix * g->dx, Y = Y0 + iy * g->dy, Z = Z0 + iz * g->dz;
    long v0, v1;
    view_window(g, Z, &v0, &v1);
    double acc = 0.0;
    for (long v = v0; v < v1; v++) {
        double beta = g->start_angle + 2.0 * M_PI * (double)v / (double)N;
        double sx = g->sid * cos(beta), sy = g->sid * sin(beta);
        double sz = g->z_start + g->feed * (double)v / (double)N;
        double ddx = X - sx, ddy = Y - sy;
        double L2 = ddx * ddx + ddy * ddy, L = sqrt(L2);
        /* the ray of fan angle gamma points along beta + gamma + pi */
        double gam = atan2(ddy, ddx) - beta - M_PI;
        gam = gam - 2.0 * M_PI * floor((gam + M_PI) / (2.0 * M_PI));
        double kf = gam / g->channel_pitch + (K - 1) / 2.0 - g->channel_offset;
        if (!(kf >= 0.0 && kf <= K - 1)) continue;
        double rf = 0.0;
        if (R > 1) {
            double w = (Z - sz) * g->sdd / L;
            rf = w / g->row_pitch + (R - 1) / 2.0 - g->row_offset;
            if (rf < 0.0) rf = 0.0;
            if (rf > R - 1) rf = R - 1;
        }
        int k0 = (int)floor(kf), r0 = (int)floor(rf);
        if (k0 > K - 2) k0 = K - 2 < 0 ? 0 : K - 2;
        if (r0 > R - 2) r0 = R - 2 < 0 ? 0 : R - 2;
        double ak = kf - k0, ar = rf - r0;
        const double *qv = q + (long)v * R * K;
        double val;
        if (R > 1) {
            double lo = (1.0 - ak) * qv[(long)r0 * K + k0] + ak * qv[(long)r0 * K + k0 + 1];
            double hi = (1.0 - ak) * qv[(long)(r0 + 1) * K + k0] + ak * qv[(long)(r0 + 1) * K + k0 + 1];
            val = (1.0 - ar) * lo + ar * hi;
        } else {
            val = (1.0 - ak) * qv[k0] + ak * qv[k0 + 1];
        }
        acc += val / L2;
    }
    return acc * dbeta;
}

/* FBP backprojection of the filtered sinogram q [V][R][K] into img [nz][ny][nx]. */
void or_fbp_backproject(const or_geometry *g, const double *q, double *img) {
    const long nvox = (long)g->nx * g->ny * g->nz;
#pragma omp parallel for schedule(dynamic, 256)
    for (long vi = 0; vi < nvox; vi++) img[vi] = fbp_voxel(g, q, vi);
}

/* The same backprojection at n listed voxels (index iz*ny*nx + iy*nx + ix) only:
 * out[i] = img[vox[i]]. */
void or_fbp_backproject_at(const or_geometry *g, const double *q, const int64_t *vox, long n, double *out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < n; i++) out[i] = fbp_voxel(g, q, vox[i]);
}

/* FBP image [nz][ny][nx] of the line-integral sinogram p [V][R][K]. */
void or_fbp(const or_geometry *g, const double *p, double *img) {
    const long n = (long)g->n_views * g->n_rows * g->n_channels;
    double *q = (double *)malloc(sizeof(double) * n);
    or_ramp_filter(g, p, q);
    or_fbp_backproject(g, q, img);
    free(q);
}

/* The "filtering" of the prior (Sec. 2.2 figure caption; reading: a separable
 * in-plane [1,2,1]/4 smoothing in x and y, edges replicated), applied n times
 * to f [nz][ny][nx] in place. */
void or_smooth_inplane(int nx, int ny, int nz, double *f, int n) {
    const long nvox = (long)nx * ny * nz;
    double *t = (double *)malloc(sizeof(double) * nvox);
    for (int pass = 0; pass < n; pass++) {
        for (long i = 0; i < nvox; i++) {
            int ix = (int)(i % nx), iy = (int)((i / nx) % ny);
            long base = i - ix - (long)iy * nx;
            double acc = 0.0;
            for (int b = -1; b <= 1; b++) {
                int y = iy + b < 0 ? 0 : (iy + b >= ny ? ny - 1 : iy + b);
                double wy = b == 0 ? 0.5 : 0.25;
                for (int a = -1; a <= 1; a++) {
                    int x = ix + a < 0 ? 0 : (ix + a >= nx ? nx - 1 : ix + a);
                    double wx = a == 0 ? 0.5 : 0.25;
                    acc += wx * wy * f[base + (long)y * nx + x];
                }
            }
            t[i] = acc;
        }
        memcpy(f, t, sizeof(double) * nvox);
    }
    free(t);
}

/* Prior image by thresholding the single-energy FBP image f. */
void or_prior(long nvox, const double *f, double t_air, double t_bone, double soft, double *prior) {
    for (long i = 0; i < nvox; i++) prior[i] = f[i] < t_air ? 0.0 : (f[i] < t_bone ? soft : f[i]);
}

/* Eq. (4): (c_1, c_2) = [[mu~_1L, mu~_2L], [mu~_1H, mu~_2H]]^-1 (mu_L, mu_H); c [nz][ny][nx][2]. */
void or_decompose(long nvox, const double *muL, const double *muH, const double calib[4], double *c) {
    double a = calib[0], b = calib[1], cc = calib[2], dd = calib[3];
    double det = a * dd - b * cc;
    for (long i = 0; i < nvox; i++) {
        c[2 * i] = (dd * muL[i] - b * muH[i]) / det;
        c[2 * i + 1] = (-cc * muL[i] + a * muH[i]) / det;
    }
}

/* The whole initialisation.  prior_in (nullable) replaces the thresholded prior
 * (so that a comparison can share the threshold decisions of another
 * implementation); prior_out, muL, muH (nullable) receive the intermediates. */
void or_mar_init(const or_geometry *g, const or_model *m, const double *d, const uint8_t *mask,
                 const or_mar_params *P, const double *prior_in, double *c, double *prior_out, double *muL,
                 double *muH) {
    const long n = (long)g->n_views * g->n_rows * g->n_channels;
    const long nvox = (long)g->nx * g->ny * g->nz;
    double *p = (double *)malloc(sizeof(double) * 2 * n);
    double *t = (double *)malloc(sizeof(double) * n);
    double *f = (double *)malloc(sizeof(double) * nvox);
    double *prior = (double *)malloc(sizeof(double) * nvox);
    double *c2 = (double *)calloc(2 * nvox, sizeof(double));
    double *l2 = (double *)malloc(sizeof(double) * 2 * n);
    double *pp = (double *)malloc(sizeof(double) * n);
    double *mL = (double *)malloc(sizeof(double) * nvox);
    double *mH = (double *)malloc(sizeof(double) * nvox);
    or_log_sinogram(g, m, d, P->count_floor, p);
    if (prior_in) {
        memcpy(prior, prior_in, sizeof(double) * nvox);
    } else {
        int j = P->prior_spectrum ? 1 : 0;
        or_complete_trace(g, p + j * n, NULL, mask, j, P->eps, t);
        or_fbp(g, t, f);
        or_smooth_inplane(g->nx, g->ny, g->nz, f, P->prior_smooth);
        or_prior(nvox, f, P->t_air, P->t_bone, P->soft_value, prior);
    }
    for (long i = 0; i < nvox; i++) c2[2 * i] = prior[i];
    or_forward(g, c2, l2, 0, g->n_views);
    for (long y = 0; y < n; y++) pp[y] = l2[2 * y];
    for (int j = 0; j < 2; j++) {
        or_complete_trace(g, p + j * n, pp, mask, j, P->eps, t);
        or_fbp(g, t, j ? mH : mL);
    }
    or_decompose(nvox, mL, mH, P->calib, c);
    if (prior_out) memcpy(prior_out, prior, sizeof(double) * nvox);
    if (muL) memcpy(muL, mL, sizeof(double) * nvox);
    if (muH) memcpy(muH, mH, sizeof(double) * nvox);
    free(p);
    free(t);
    free(f);
    free(prior);
    free(c2);
    free(l2);
    free(pp);
    free(mL);
    free(mH);
}
