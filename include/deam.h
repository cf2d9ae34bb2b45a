/*
 * deam.h -- C ABI of the GB300 (sm_103a) MAR-DEAM library (libdeam.so).
 *
 * MAR-DEAM (Ge et al., "A Metal Artifact Reduction Scheme For Accurate Iterative
 * Dual-Energy CT Algorithms", arXiv 2202.00116) reconstructs two basis-component
 * images c_1, c_2 from low- and high-kVp transmission data d_L, d_H by dual-energy
 * alternating minimisation (DEAM) of the I-divergence (Sec. 2.3, Eq. 5) between the
 * data and the polyenergetic forward model
 *     g_j(y:c) = sum_E I0_j(y,E) exp(-sum_x h(x,y) sum_i mu_i(E) c_i(x))   (Eq. 8),
 * where every ray on the metal trace T(y) = sum_x h(x,y) M(x) >= t has its data
 * replaced by the current estimate (Eqs. 2-3 and 11: p_j(y,E) = q_j(y,E) there).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Images are float32 [nz][ny][nx][2]: the two basis components interleaved
 *    (c_1, c_2) per voxel.  Ray arrays are [n_views][n_rows][n_channels], with a
 *    trailing pair for two-component ray data.  Measured data is float32
 *    [2][n_views][n_rows][n_channels] counts, j = 0 (low kVp), 1 (high kVp).
 *  * Geometry (third-generation helical CT, curved detector):
 *      source of view v at angle beta_v = start_angle + 2 pi v / views_per_rotation,
 *        s_v = (sid cos beta_v, sid sin beta_v, z_start + feed v / views_per_rotation);
 *      channel k at fan angle gamma_k = (k - (K-1)/2 + channel_offset) channel_pitch;
 *      row r at height w_r = (r - (R-1)/2 + row_offset) row_pitch (mm at the detector);
 *      ray (v,r,k) leaves s_v along u = (-sdd cos(beta_v+gamma_k), -sdd sin(beta_v+gamma_k), w_r);
 *      voxel (ix,iy,iz) is centred at (cx + (ix-(nx-1)/2) dx, cy + ..., cz + ...).
 *    The volume must lie strictly inside the source circle.
 *  * h(x,y) is Joseph's method: one sample per voxel-centre plane of the dominant
 *    transaxial axis (x when |u_x| >= |u_y|), bilinear in the other two axes,
 *    weight (plane spacing) |u| / |u_dominant|; taps outside the volume are zero.
 *  * `stream` is a cudaStream_t (NULL = the legacy default stream).  All work is
 *    enqueued on it; calls that return host values synchronise it.
 *  * Device pointers are borrowed for the duration of the call.  Where a parameter
 *    says "host or device", a host pointer is detected with cudaPointerGetAttributes
 *    and staged through the context's device buffers.
 *  * Every call returns DEAM_OK or an error code; deam_last_error() gives a
 *    message for the calling thread.  Arguments are validated on the host before
 *    any launch.  A CUDA error leaves the context unusable (DEAM_ERR_STATE).
 */
#ifndef DEAM_H
#define DEAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    DEAM_OK = 0,
    DEAM_ERR_ARG = 1,     /* invalid argument or geometry */
    DEAM_ERR_CUDA = 2,    /* a CUDA runtime call or kernel failed */
    DEAM_ERR_OOM = 3,     /* device allocation failed */
    DEAM_ERR_STATE = 4,   /* call not valid in the context's state (no data, earlier failure) */
    DEAM_ERR_TIMEOUT = 5, /* a bounded device wait expired (reserved: no kernel here waits on
                             another block, a flag or a peer, so none is returned) */
    DEAM_ERR_NUMERIC = 6  /* non-finite objective */
};

enum { DEAM_GEOM_FAN2D = 0, DEAM_GEOM_HELICAL = 1 };

enum {
    DEAM_MASK_VOXEL_IMAGE = 0,       /* m: float32 metal image M [nz][ny][nx]; mask = (A M >= t), both spectra */
    DEAM_MASK_RAY = 1,               /* m: uint8 [V][R][K], nonzero = metal-trace ray for both spectra */
    DEAM_MASK_RAY_PER_SPECTRUM = 2   /* m: uint8 [V][R][K], bit 0: on the trace T_L of the low-kVp data,
                                        bit 1: on the trace T_H of the high-kVp data (Sec. 2.1) */
};

/* Scanner and volume geometry (lengths in mm, angles in rad). */
typedef struct deam_geometry {
    int kind; /* DEAM_GEOM_FAN2D (n_rows = 1, feed = 0) or DEAM_GEOM_HELICAL */
    int nx, ny, nz;
    double dx, dy, dz;
    double cx, cy, cz; /* volume centre */
    double sid, sdd;   /* source-isocentre and source-detector distances */
    int n_views, views_per_rotation;
    double start_angle, feed, z_start; /* feed = table travel per rotation */
    int n_rows;
    double row_pitch; /* at the detector */
    int n_channels;
    double channel_pitch; /* fan angle between channels */
    double channel_offset, row_offset; /* detector shifts, in cells */
} deam_geometry;

/* Source spectra I0_j(y,E) = I0[j][E] * bowtie[channel] (Eq. 8: "contains the
 * spectrum and the bowtie filter").  Bins where both spectra are zero are skipped. */
typedef struct deam_spectra {
    int n_e;                 /* energy bins, 1..256 */
    const double *energy_keV; /* [n_e] bin centres (informational, may be NULL) */
    const double *I0;        /* [2][n_e] counts per ray per bin, >= 0 */
    const double *bowtie;    /* [n_channels] factors > 0, or NULL for 1 */
} deam_spectra;

/* Basis attenuation mu_i(E) of the two components, 1/mm, >= 0 (Eq. 8). */
typedef struct deam_basis {
    int n_e;
    const double *mu; /* [2][n_e] */
} deam_basis;

typedef struct deam_options {
    double metal_threshold; /* t of Sec. 2.1 in mm of metal path; <= 0: half the smallest voxel edge */
    double Z;               /* c-step normaliser; <= 0: max_E(mu_1+mu_2) * max_y sum_x h(x,y) */
    double penalty_lambda;  /* lambda of Eq. (6); 0 (default): unregularised MAR-DEAM */
    double penalty_delta;   /* delta of Eq. (7) (> 0 when lambda > 0) */
    int clamp_nonneg;       /* 1: clamp c_i >= 0 after each c-step (the paper is silent; default 0) */
    int precision;          /* 0 (default): spectral sums in compensated FP32 and the objective in FP64;
                               1: plain FP32 sums and FP32 objective accumulation (for comparison).
                               Projection sampling is FP32 either way.  A batch holding a context
                               with 1 runs its per-scan plan only (the persistent plan has only 0). */
    int reserved[6];        /* zero */
} deam_options;

typedef struct deam_ctx deam_ctx;

/* Create a context for one scan: validates the geometry, copies the spectra and
 * attenuation tables to the current CUDA device, allocates the context's device
 * buffers (measurements, metal mask, per-ray payload, reduction partials, the
 * projector's volume layouts) and computes the normaliser Z (Appendix-style
 * surrogate condition sum_{x,i} h mu_i / Z <= 1 for every ray and active bin).
 * opts may be NULL for defaults.  Returns DEAM_ERR_ARG, DEAM_ERR_OOM or
 * DEAM_ERR_CUDA on failure (*out is then NULL). */
int deam_init(const deam_geometry *geom, const deam_spectra *spectra, const deam_basis *basis,
              const deam_options *opts, deam_ctx **out);

/* Store the measurements d (host or device, float32 [2][V][R][K], counts) as the
 * nonnegative substitution d~ = max(d, 0) (Sec. 2.1).  A host buffer may be
 * reused as soon as the call returns (the call waits for its copy); a device
 * buffer is read on `stream`. */
int deam_set_data(deam_ctx *ctx, const float *d, void *stream);

/* Set the metal trace (Sec. 2.1: rays with T(y) >= t are "metal").  kind =
 * DEAM_MASK_VOXEL_IMAGE: m is the metal image M (host or device float32
 * [nz][ny][nx]), forward-projected on the GPU and thresholded at opts.metal_threshold
 * (T = t counts as metal) for both spectra.  kind = DEAM_MASK_RAY: m is a uint8
 * ray mask (host or device), nonzero = metal for both spectra.  kind =
 * DEAM_MASK_RAY_PER_SPECTRUM: separate traces T_L, T_H as bits 0 and 1 (for
 * scans whose two spectra see different system operators, e.g. motion between
 * the acquisitions); the substitution p = q then applies per spectrum.  Until
 * called, no ray is metal (plain DEAM). */
int deam_set_metal_mask(deam_ctx *ctx, const void *m, int kind, void *stream);

/* Copy the current metal mask (uint8 [V][R][K], bit j = on the trace of
 * spectrum j) to device memory `mask`. */
int deam_get_metal_mask(deam_ctx *ctx, uint8_t *mask, void *stream);

/* Forward model at image c (device float32 [nz][ny][nx][2]): line integrals
 * l_i(y) = sum_x h(x,y) c_i(x) into l (device float32 [V][R][K][2], may be NULL)
 * and, if g is not NULL, the expected counts g_j(y:c) of Eq. (8) into g (device
 * float32 [2][V][R][K]). */
int deam_forward(deam_ctx *ctx, const float *c, float *l, float *g, void *stream);

/* Adjoint of the projector: img_i(x) = sum_y h(x,y) y_i(y), exactly the transpose
 * of deam_forward's h.  y: device float32 [V][R][K][2]; img: device float32
 * [nz][ny][nx][2], overwritten.  Gather form: deterministic, no atomics. */
int deam_backproject(deam_ctx *ctx, const float *y, float *img, void *stream);

/* Per-ray quantities of one MAR-DEAM iteration at image c (device): payload
 * (device float32 [V][R][K][4]) = (B~_1, B~_2, D_1, D_2) with
 * B~_i = sum_j S_ij, D_i = sum_j (r_j - 1) S_ij, S_ij = sum_E mu_i(E) q_j(y,E),
 * r_j = d~_j/g_j off the metal trace and 1 on it (Eqs. 9-11); *F (host, may be
 * NULL) receives the objective of deam_objective.  Needs deam_set_data. */
int deam_ray_terms(deam_ctx *ctx, const float *c, float *payload, double *F, void *stream);

/* Run n_iter MAR-DEAM iterations in place on c (host or device float32
 * [nz][ny][nx][2]).  Each iteration: forward projection with the fused spectral
 * sums, metal-trace substitution and p-step ratio; the objective
 * F(c^k) = sum_j sum_{T(y)<t} I(d~_j || g_j(c^k)) (Eq. 5 with Eqs. 2-3) into
 * hist[k] (host, may be NULL); then the gather backprojection of the payload fused
 * with the c-step c_i <- c_i - (1/Z) ln(b^_i / b~_i), where b~_i = sum_{y,E} h mu_i q
 * and b^_i = sum_{y,E} h mu_i p (computed as log1p(delta_i / b~_i) with
 * delta_i = b^_i - b~_i backprojected directly).  Voxels with b~_i <= 0 or
 * b^_i <= 0 are left unchanged.  Needs deam_set_data.  Deterministic. */
int deam_iterate(deam_ctx *ctx, float *c, int n_iter, double *hist, void *stream);

/* F(c) (Eq. 5 over rays off the metal trace) into *out (host). Needs deam_set_data. */
int deam_objective(deam_ctx *ctx, const float *c, double *out, void *stream);

/* Gradient of the objective with respect to the image (derivative of Eq. 5
 * through Eq. 8, metal-trace rays excluded): dF/dc_i(x) = b^_i(x) - b~_i(x) =
 * sum_y h(x,y) sum_j (r_j - 1) S_ij(y), written to grad (device float32
 * [nz][ny][nx][2], overwritten).  The per-ray terms are recomputed from c
 * (nothing per energy bin is stored); *F (host, may be NULL) receives F(c).
 * Needs deam_set_data.  Deterministic. */
int deam_gradient(deam_ctx *ctx, const float *c, float *grad, double *F, void *stream);

/* The two backprojected sums of the c-step (Sec. 2.3 update, derived from
 * Eqs. 5 and 8-11) at c, without applying it: sums (device float32
 * [nz][ny][nx][4], overwritten) receives per voxel (b~_1, b~_2, delta_1,
 * delta_2), b~_i = sum_{y,E} h mu_i q and delta_i = b^_i - b~_i (= dF/dc_i).
 * The c-step would be c_i - (1/Z) log1p(delta_i / b~_i); -delta_i / (Z b~_i)
 * is the diagonally preconditioned gradient step it approximates.  *F (host,
 * may be NULL) receives F(c); *Z (host, may be NULL) the context's Z.  Needs
 * deam_set_data.  Deterministic. */
int deam_backprojected_sums(deam_ctx *ctx, const float *c, float *sums, double *F, double *Z, void *stream);

/* ---- MAR initialisation (Sec. 2.2 and Eq. 4) ---------------------------------
 * The starting image c^0 of MAR-DEAM: the measured sinograms of both spectra
 * are completed across their metal traces by normalised metal-artifact
 * reduction (NMAR: divide by the forward projection of a prior image,
 * interpolate linearly along the channels, multiply back), reconstructed by
 * filtered backprojection, and split into the basis components by the
 * image-domain decomposition of Eq. (4).  The prior thresholds a
 * single-energy FBP image, filtered (Sec. 2.2: the prior is obtained by
 * thresholding and filtering).
 * FBP: equiangular fan-beam filtered backprojection on the curved detector
 * (pre-weight SID cos(gamma), the discrete equiangular ramp kernel), extended
 * to the helix FDK-style (cone pre-weight SDD / sqrt(SDD^2 + w^2); each voxel
 * takes the one rotation of views centred on the view whose source z equals
 * its own, rows interpolated at w = (z - z_s) SDD / L and clamped to the end
 * rows; channels outside the detector contribute nothing).  All need
 * deam_set_data; trace completion needs the metal mask.  Work is enqueued on
 * `stream`; scratch is allocated per call (these run once per scan). */
typedef struct deam_mar_params {
    double calib[4];       /* mu~_1L, mu~_2L, mu~_1H, mu~_2H of Eq. (4): FBP value (1/mm) of unit c_i
                              in the spectrum-j image; the 2x2 matrix must be invertible */
    double t_air;          /* prior: FBP values below -> 0 (1/mm) */
    double t_bone;         /* prior: values at or above are kept (1/mm) */
    double soft_value;     /* prior: value of voxels in [t_air, t_bone) (1/mm) */
    double count_floor;    /* counts: d~ is floored here before the log (> 0; 1 is typical) */
    double eps;            /* NMAR: the prior projection is floored here before dividing (> 0) */
    int prior_spectrum;    /* single-energy image of the prior: 0 = L, 1 = H */
    int prior_smooth;      /* passes (0..16) of an in-plane [1,2,1]/4 x [1,2,1]/4 smoothing of that
                              image before the thresholds (the prior's "filtering"; edges replicated) */
    int reserved[6];       /* zero */
} deam_mar_params;

/* Line-integral sinograms p_j(y) = ln(I0_j(y) / max(d~_j(y), count_floor)),
 * I0_j(y) = sum_E I0_j(E) bowtie(k).  p: device float32 [2][V][R][K]. */
int deam_log_sinogram(deam_ctx *ctx, double count_floor, float *p, void *stream);

/* Trace completion of one sinogram p (device float32 [V][R][K]) into out (same
 * shape; may equal p) over the rays whose mask bit `spectrum` (0 = L, 1 = H) is
 * set: linear interpolation along the channels of each (view, row) between the
 * nearest rays off the trace (constant beyond the row's ends).  With prior_proj
 * (device float32 [V][R][K], the prior image's projection) the interpolated
 * quantity is p / max(prior_proj, eps), multiplied back afterwards (NMAR);
 * with NULL it is p itself.  Rays off the trace are copied unchanged. */
int deam_complete_trace(deam_ctx *ctx, const float *p, const float *prior_proj, int spectrum, double eps,
                        float *out, void *stream);

/* FBP images img[i] (device float32 [n][nz][ny][nx], 1/mm) of n = 1 or 2
 * line-integral sinograms p[i] (device float32 [n][V][R][K]).  FBP (here and in
 * deam_mar_init) supports 2 to 3072 channels; more return DEAM_ERR_ARG. */
int deam_fbp(deam_ctx *ctx, const float *p, int n, float *img, void *stream);

/* The whole initialisation into c (device float32 [nz][ny][nx][2]).  prior_in
 * (nullable, device float32 [nz][ny][nx]) replaces the thresholded prior;
 * prior_out (nullable, same shape) receives the prior used; mu_out (nullable,
 * device float32 [2][nz][ny][nx]) the two NMAR-corrected FBP images. */
int deam_mar_init(deam_ctx *ctx, const deam_mar_params *params, const float *prior_in, float *c, float *prior_out,
                  float *mu_out, void *stream);

/* Linear images of the basis components (Sec. 3): out[e] = a_e c_1 + b_e c_2 for
 * n coefficient pairs coef[2e] = a_e, coef[2e+1] = b_e (host, 1 <= n <= 256).
 * With (a_e, b_e) = (mu_1(E_e), mu_2(E_e)) these are virtual monoenergetic
 * images mu(x, E) (paper Fig. 5: 20, 60, 140 keV); with (a, b) = sum_E w_j(E)
 * (mu_1(E), mu_2(E)), w_j the normalised spectrum j, they are the
 * spectrum-weighted averages of the VMIs shown as 90 and 140 kVp images.
 * c: device float32 [nz][ny][nx][2]; out: device float32 [n][nz][ny][nx].
 * Synchronises `stream`. */
int deam_basis_images(deam_ctx *ctx, const float *c, const double *coef, int n, float *out, void *stream);

/* Virtual monoenergetic images (Sec. 3, Fig. 5) at n energies (host, keV,
 * 1 <= n <= 256): out[e] = mu_1(E_e) c_1 + mu_2(E_e) c_2 (1/mm), mu_i(E) taken
 * from the context's basis tables by linear interpolation of ln mu_i between
 * the bin centres (the end values beyond them).  Needs the bin energies at
 * deam_init (DEAM_ERR_STATE without).  c: device float32 [nz][ny][nx][2]; out:
 * device float32 [n][nz][ny][nx].  Synchronises `stream`. */
int deam_vmi(deam_ctx *ctx, const float *c, const double *energies, int n, float *out, void *stream);

/* The two spectrum-weighted averages of the VMIs (Sec. 3: the 90 and 140 kVp
 * images): out[j] = sum_E w_j(E) (mu_1(E) c_1 + mu_2(E) c_2) with
 * w_j = I0_j / sum_E I0_j, j = 0 (low kVp), 1 (high kVp).  out: device float32
 * [2][nz][ny][nx].  Synchronises `stream`. */
int deam_kvp_images(deam_ctx *ctx, const float *c, float *out, void *stream);

/* The penalty R(c) of Eqs. (6)-(7) with the context's lambda and delta into *R
 * (host): R = lambda sum_i sum_x sum_{x~ in N_x} w(x,x~) phi(c_i(x) - c_i(x~)),
 * N_x the 26 neighbours inside the volume, w = 1/physical distance,
 * phi(u) = delta^2 (|u|/delta - log(1 + |u|/delta)) (the convex reading of the
 * garbled Eq. 7).  With lambda > 0, deam_iterate's c-step minimises the DEAM
 * surrogate plus De Pierro's separable surrogate of R per voxel, so F + R does
 * not increase; voxels no data reaches are then moved by the penalty alone.
 * c: device float32 [nz][ny][nx][2]. */
int deam_penalty(deam_ctx *ctx, const float *c, double *R, void *stream);

/* Normaliser Z in use, and the number of (voxel, component) pairs left unchanged
 * by the last c-step (b~ <= 0 or b^ <= 0). Either pointer may be NULL. */
int deam_info(deam_ctx *ctx, double *Z, long long *skipped_last);

/* Number of Joseph samples (ray, plane) pairs with at least one tap in the
 * volume, summed over all rays: the work of one projection (host *n). */
int deam_count_samples(deam_ctx *ctx, long long *n, void *stream);

/* Bounds-checked builds.  A library compiled with -DDEAM_BOUNDS_CHECK (the
 * build script's bounds_check option: libdeam_checked.so) tests the index of
 * every guarded device access in the projector kernels first; a failing test
 * records the site and index in the context's fault words (the first one
 * only), skips the access and never traps, and the entry point reads the words
 * back on return (synchronising its stream) and returns DEAM_ERR_ARG with the
 * site in deam_last_error().  deam_bounds_checked() is 1 in such a build, else
 * 0.  deam_bounds_inject(ctx) writes a fault record from the host (no device
 * fault is made), so that the next entry point reports it: a test of the
 * read-back path; DEAM_ERR_STATE in an unchecked build. */
int deam_bounds_checked(void);
int deam_bounds_inject(deam_ctx *ctx, void *stream);

/* Measured load throughput (bytes/s, into *bytes_per_s, host) of the current
 * device's L1 data path, the on-chip unit that bounds the projector's gathers:
 * every SM streams conflict-free 16-byte shared-memory loads for a few
 * milliseconds, timed with CUDA events on `stream` (best of three after a
 * warm-up run).  Changes no device setting.  Synchronises `stream`. */
int deam_l1_bandwidth(double *bytes_per_s, void *stream);

/* Per-kernel timing of deam_iterate.  enable = 1 records CUDA events on the
 * call's stream around every kernel of every iteration (layout build, forward +
 * epilogue, objective reduction, backprojection + update) and accumulates their
 * durations; enable = 0 stops.  deam_kernel_times copies the accumulated
 * milliseconds and launch counts of those four stages into ms[4] and
 * launches[4] (either may be NULL) and, if reset is nonzero, clears them. */
int deam_profile(deam_ctx *ctx, int enable);
int deam_kernel_times(deam_ctx *ctx, double *ms, long long *launches, int reset);

/* ---- Batched scans ------------------------------------------------------
 * Many independent scans of uneven size and view count, iterated together.
 * Each scan is a context from deam_init with deam_set_data (and optionally
 * deam_set_metal_mask) called; contexts must outlive the batch, live on the
 * current device, and not be used by other calls while the batch iterates.
 * One iteration of the batch is the MAR-DEAM iteration of deam_iterate for
 * every scan, run as one persistent forward launch and one persistent
 * backprojection launch over the work of all scans, captured once in a CUDA
 * graph and replayed.  autotune = 0 runs the persistent plan with default
 * shapes, 2 the per-scan plan (below) without tuning.  With autotune = 1 the first deam_batch_iterate times the
 * candidate ray-tile shapes (32 channels x rows x views) and backprojection
 * shapes (z-slab depth x column tile) on scratch copies of the images and keeps
 * the fastest, then times one iteration of that persistent plan against a plan
 * that replays every scan's own kernels on parallel graph branches, and keeps
 * the faster plan; results equal deam_iterate's up to FP32 summation order. */
typedef struct deam_batch deam_batch;

int deam_batch_create(deam_ctx *const *ctxs, int n, int autotune, deam_batch **out);

/* n_iter iterations of every scan in place on its image c[i] (device float32
 * [nz][ny][nx][2], one per context, in creation order).  hist (host, may be
 * NULL) receives F(c_i^k) at hist[i * n_iter + k].  Synchronises `stream`.
 * The graph is re-captured when the image pointers change. */
int deam_batch_iterate(deam_batch *b, float *const *c, int n_iter, double *hist, void *stream);

/* Execution plan: *plan = 0 (persistent launches over all scans) or 1 (each
 * scan's own kernels on a graph branch of its own), plan_ms[2] = the tuning
 * time of one captured iteration of each plan.  Chosen shapes of the
 * persistent plan: fwd_shape[2] = (rows, views) of the forward ray tile;
 * bwd_shapes[3][3] = (slab depth, tile x, tile y) for the slab classes 2, 8 and
 * 16 (a scan's class follows its geometry; zeros where no scan falls in a
 * class: each non-empty class gets its own persistent launch); fwd_ms[3],
 * bwd_ms[6] = the tuning times of every candidate (0 if not tuned).  Any
 * pointer may be NULL. */
int deam_batch_info(deam_batch *b, int *plan, float *plan_ms, int *fwd_shape, int *bwd_shapes, float *fwd_ms,
                    float *bwd_ms);

int deam_batch_destroy(deam_batch *b);

/* F(c) as deam_objective computes it, for callers that cannot allocate device
 * memory and so cannot create a context (deam_init allocates its buffers): code
 * running where device memory belongs to another allocator or a fixed arena, or
 * in a latency-bound loop where cudaMalloc/cudaFree would synchronise the device.
 * The paper has no counterpart; this is a library-usage variant.
 * The geometry, spectra and basis are checked exactly as deam_init checks them
 * (DEAM_ERR_ARG on refusal).
 * Inputs are caller-owned device buffers: c float32 [nz][ny][nx][2], d float32
 * [2][V][R][K] raw counts (clamped to >= 0 on the fly), mask uint8 [V][R][K] or
 * NULL (no metal).  The mask is read as deam_get_metal_mask writes it: bit 0
 * leaves out the ray's low-kVp term, bit 1 its high-kVp term (Sec. 2.1, Eq. 11),
 * so a plain 0/1 mask meant for both spectra must be given as 0/3.  Output F is
 * one device double, written on `stream`; it may be +inf or NaN (a ray with
 * counts but zero expected counts, or non-finite inputs), which deam_objective
 * reports as DEAM_ERR_NUMERIC but this call cannot see without reading F back:
 * the caller checks it.  Nothing
 * is allocated: the only scratch (one FP64 partial per 128 rays) is a static
 * 8 MiB device array that every GPU loading the library holds until exit, so at
 * most 134,217,728 rays (more: DEAM_ERR_ARG); a bowtie may have at most 1024
 * channels.  The first call on a device looks up that array's device address
 * (set-up): make it before any stream capture.  All calls share the array, so
 * calls that overlap on the GPU race: serialise them. */
int deam_objective_noalloc(const deam_geometry *geom, const deam_spectra *spectra, const deam_basis *basis,
                           const float *c, const float *d, const uint8_t *mask, double *F, void *stream);

/* Release the context and its device buffers (waits for its work). NULL is a no-op.
 * A context held by a live batch is not released: DEAM_ERR_STATE (destroy the
 * batch first). */
int deam_destroy(deam_ctx *ctx);

/* Message of the last error on the calling thread ("" if none). */
const char *deam_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DEAM_H */
