// C ABI of the sm_103a MAR-DEAM library: argument validation, geometry tables,
// device buffers and the launch sequence of each entry point (see include/deam.h).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "deam.h"
#include "deam_ctx.h"
#include "deam_internal.h"

using deam::Geo;
using deam::Spec;
using deam::build_layouts;
using deam::fwd_args;
using deam::slab_view_range;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

const double kPi = 3.14159265358979323846;

bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// NVTX range around the host-side enqueue of one stage (named in a profiler's
// timeline; free when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

int deam::set_error(int code, const char* msg) { return fail(code, msg); }



#define CK(x)                                                                                  \
    do {                                                                                       \
        cudaError_t e_ = (x);                                                                  \
        if (e_ != cudaSuccess) {                                                               \
            ctx->failed = true;                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? DEAM_ERR_OOM : DEAM_ERR_CUDA,        \
                        std::string(#x) + ": " + cudaGetErrorString(e_));                      \
        }                                                                                      \
    } while (0)

// Device-only arguments are checked on the host: a host pointer would otherwise
// fail inside the runtime or fault in a kernel and leave the context unusable.
#define NEED_DEVICE(p, name)                                                         \
    do {                                                                             \
        if ((p) && !is_device_ptr(p)) return fail(DEAM_ERR_ARG, name " must be device memory"); \
    } while (0)

#define CHECK_CTX(ctx)                                                              \
    do {                                                                            \
        if (!(ctx)) return fail(DEAM_ERR_ARG, "null context");                      \
        if ((ctx)->failed) return fail(DEAM_ERR_STATE, "context failed earlier"); \
    } while (0)

// End of an entry point that launched kernels: in a bounds-checked build the
// context's fault words are read back (synchronising `s`) and a recorded
// out-of-range access is reported as DEAM_ERR_ARG (and cleared); otherwise
// DEAM_OK without touching the stream.
int deam::finish_call(deam_ctx* ctx, cudaStream_t s) {
#ifdef DEAM_BOUNDS_CHECK
    unsigned int w[2] = {0, 0};
    CK(cudaMemcpyAsync(w, ctx->fault, sizeof(w), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (w[0] != 0) {
        CK(cudaMemsetAsync(ctx->fault, 0, sizeof(w), s));
        CK(cudaStreamSynchronize(s));
        char m[160];
        snprintf(m, sizeof(m), "bounds check: out-of-range access at site %u (index %u)", w[0], w[1]);
        return fail(DEAM_ERR_ARG, m);
    }
#else
    (void)ctx;
    (void)s;
#endif
    return DEAM_OK;
}

template <typename T>
static cudaError_t dalloc(T** p, size_t n) {
    return cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(n, 1));
}

static void free_ctx(deam_ctx* c) {
    void* ptrs[] = {c->view4, c->view_z, c->ip4, c->ipL, c->chan, c->row, c->bowtie, c->dt, c->mask, c->payload,
                    c->volX, c->volY, c->partial, c->scal, c->hist, c->slab_views, c->skipped, c->c_stage,
                    c->coef, c->sums, c->fault};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete c;
}

// Host-side validation of a scan description, shared by deam_init and the
// context-free entry point: "" when valid, else the reason.
std::string deam::validate_scan(const deam_geometry* g, const deam_spectra* s, const deam_basis* b) {
    if (!g || !s || !b) return "geometry, spectra and basis must not be NULL";
    if (g->kind != DEAM_GEOM_FAN2D && g->kind != DEAM_GEOM_HELICAL) return "geometry.kind must be FAN2D or HELICAL";
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return "volume dimensions must be >= 1";
    if (!finite_pos(g->dx) || !finite_pos(g->dy) || !finite_pos(g->dz)) return "voxel sizes must be finite and > 0";
    if (!isfinite(g->cx) || !isfinite(g->cy) || !isfinite(g->cz)) return "volume centre must be finite";
    if (!finite_pos(g->sid) || !finite_pos(g->sdd) || g->sdd <= g->sid) return "need 0 < sid < sdd";
    if (g->n_views < 1 || g->views_per_rotation < 1) return "n_views and views_per_rotation must be >= 1";
    if (g->n_rows < 1 || g->n_channels < 1) return "detector must have >= 1 row and channel";
    if (!finite_pos(g->channel_pitch)) return "channel_pitch must be finite and > 0";
    if (g->n_rows > 1 && !finite_pos(g->row_pitch)) return "row_pitch must be finite and > 0";
    if (!isfinite(g->start_angle) || !isfinite(g->feed) || !isfinite(g->z_start) || !isfinite(g->channel_offset) ||
        !isfinite(g->row_offset) || !isfinite(g->row_pitch))
        return "geometry values must be finite";
    if (g->kind == DEAM_GEOM_FAN2D && (g->n_rows != 1 || g->feed != 0.0))
        return "FAN2D geometry needs n_rows = 1 and feed = 0";
    if ((double)g->channel_pitch * g->n_channels >= kPi) return "fan wider than pi";
    // the volume (plus one voxel of interpolation support) must lie inside the source circle
    double rmax = 0.0;
    for (int sx = -1; sx <= 1; sx += 2)
        for (int sy = -1; sy <= 1; sy += 2) {
            double x = g->cx + sx * (g->nx + 1) / 2.0 * g->dx, y = g->cy + sy * (g->ny + 1) / 2.0 * g->dy;
            rmax = std::max(rmax, sqrt(x * x + y * y));
        }
    if (rmax >= 0.98 * g->sid) return "volume must lie inside the source circle";
    // 32-bit index limits of the kernels
    const double big = 2147483647.0;
    if ((double)g->nx * (g->nz + 2) * (g->ny + 1) >= big || (double)g->ny * (g->nz + 2) * (g->nx + 1) >= big)
        return "volume too large for 32-bit plane indexing";
    if ((double)g->n_views * g->n_rows >= big) return "too many views x rows";
    if (s->n_e < 1 || s->n_e > deam::kMaxE) return "spectra.n_e must be in [1, 256]";
    if (b->n_e != s->n_e) return "basis.n_e must equal spectra.n_e";
    if (!s->I0 || !b->mu) return "spectra.I0 and basis.mu must not be NULL";
    bool any = false;
    for (int i = 0; i < 2 * s->n_e; ++i) {
        if (!isfinite(s->I0[i]) || s->I0[i] < 0.0) return "I0 must be finite and >= 0";
        if (!isfinite(b->mu[i]) || b->mu[i] < 0.0) return "mu must be finite and >= 0";
        any = any || s->I0[i] > 0.0;
    }
    if (!any) return "both spectra are empty";
    if (s->bowtie)
        for (int k = 0; k < g->n_channels; ++k)
            if (!finite_pos(s->bowtie[k])) return "bowtie factors must be finite and > 0";
    return "";
}

// View range [lo, hi] whose rays can put a sample into the z-range of slab s
// (voxel centres +- one slice of interpolation support) at the columns
// [ix0, ix1] x [iy0, iy1].  A sample tapping those columns lies within one voxel
// of them, at most rmax from the rotation axis, so its ray parameter t (the
// fraction of the source-detector distance) is within (sid -+ rmax) / sdd and its
// height is s_z + t w for the ray's row height w at the detector.
int2 deam::slab_view_range(const deam_geometry& g, int s, int slab, int ix0, int ix1, int iy0, int iy1) {
    const int z0 = s * slab, z1 = std::min(g.nz, z0 + slab) - 1;
    if (g.feed == 0.0 || g.nz == 1) return make_int2(0, g.n_views - 1);
    const double Z0 = g.cz - (g.nz - 1) / 2.0 * g.dz;
    const double zlo = Z0 + (z0 - 1) * g.dz, zhi = Z0 + (z1 + 1) * g.dz;
    const double X0 = g.cx - (g.nx - 1) / 2.0 * g.dx, Y0 = g.cy - (g.ny - 1) / 2.0 * g.dy;
    double rmax = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const double x = X0 + (a ? ix1 + 1 : ix0 - 1) * g.dx, y = Y0 + (b ? iy1 + 1 : iy0 - 1) * g.dy;
            rmax = std::max(rmax, sqrt(x * x + y * y));
        }
    const double t0 = (g.sid - rmax) / g.sdd, t1 = (g.sid + rmax) / g.sdd;
    const double w0 = (0 - (g.n_rows - 1) / 2.0 + g.row_offset) * g.row_pitch;
    const double w1 = (g.n_rows - 1 - (g.n_rows - 1) / 2.0 + g.row_offset) * g.row_pitch;
    const double tw[4] = {t0 * w0, t0 * w1, t1 * w0, t1 * w1};
    const double twmax = *std::max_element(tw, tw + 4), twmin = *std::min_element(tw, tw + 4);
    // z* = s_z + t w  in [zlo, zhi]  <=>  s_z in [zlo - max(t w), zhi - min(t w)]
    const double szlo = zlo - twmax, szhi = zhi - twmin;
    double va = (szlo - g.z_start) * g.views_per_rotation / g.feed;
    double vb = (szhi - g.z_start) * g.views_per_rotation / g.feed;
    if (va > vb) std::swap(va, vb);
    long long lo = (long long)floor(va) - 2, hi = (long long)ceil(vb) + 2;
    lo = std::max(lo, 0LL);
    hi = std::min(hi, (long long)g.n_views - 1);
    if (lo > hi) return make_int2(1, 0);
    return make_int2((int)lo, (int)hi);
}

std::vector<int2> deam::tile_view_ranges(const deam_geometry& g, int slab, int tx, int ty) {
    const int ntx = (g.nx + tx - 1) / tx, nty = (g.ny + ty - 1) / ty, ns = (g.nz + slab - 1) / slab;
    std::vector<int2> v;
    v.reserve((size_t)ntx * nty * ns);
    for (int z = 0; z < ns; ++z)
        for (int by = 0; by < nty; ++by)
            for (int bx = 0; bx < ntx; ++bx)
                v.push_back(slab_view_range(g, z, slab, bx * tx, std::min(g.nx, (bx + 1) * tx) - 1, by * ty,
                                            std::min(g.ny, (by + 1) * ty) - 1));
    return v;
}

int deam::build_layouts(deam_ctx* ctx, const float2* c, const float* m, int ones, cudaStream_t s) {
    CK(deam::launch_layout(c, m, ones, ctx->volX, ctx->volY, ctx->geo.nx, ctx->geo.ny, ctx->geo.nz, s));
    return DEAM_OK;
}

deam::FwdArgs deam::fwd_args(deam_ctx* ctx) {
    deam::FwdArgs A{};
    A.volX = ctx->volX;
    A.volY = ctx->volY;
    A.bowtie = ctx->bowtie;
    A.partial = ctx->partial;
    return A;
}

void deam::set_penalty_args(const deam_ctx* ctx, BwdArgs& B) {
    B.sums = ctx->lambda > 0.0 ? ctx->sums : nullptr;
    B.lambda = (float)ctx->lambda;
    B.delta = (float)ctx->delta;
    B.Z = (float)ctx->Z;
    B.pdx = (float)ctx->geo.dx;
    B.pdy = (float)ctx->geo.dy;
    B.pdz = (float)ctx->geo.dz;
    B.volX = ctx->volX;
}

extern "C" {

const char* deam_last_error(void) { return g_err.c_str(); }

int deam_init(const deam_geometry* geom, const deam_spectra* spectra, const deam_basis* basis,
              const deam_options* opts, deam_ctx** out) {
    if (!out) return fail(DEAM_ERR_ARG, "out must not be NULL");
    *out = nullptr;
    std::string why = deam::validate_scan(geom, spectra, basis);
    if (!why.empty()) return fail(DEAM_ERR_ARG, why);
    deam_options o{};
    if (opts) o = *opts;
    if (!isfinite(o.metal_threshold) || !isfinite(o.Z) || !isfinite(o.penalty_lambda) || !isfinite(o.penalty_delta))
        return fail(DEAM_ERR_ARG, "options must be finite");
    if (o.penalty_lambda < 0.0 || (o.penalty_lambda > 0.0 && !(o.penalty_delta > 0.0)))
        return fail(DEAM_ERR_ARG, "need penalty_lambda >= 0 and penalty_delta > 0 when penalty_lambda > 0");

    deam_ctx* ctx = new deam_ctx();
    const deam_geometry& g = *geom;
    ctx->geo = g;
    if (cudaGetDevice(&ctx->device) != cudaSuccess) {
        delete ctx;
        return fail(DEAM_ERR_CUDA, "no CUDA device");
    }
    ctx->nrays = (long long)g.n_views * g.n_rows * g.n_channels;
    ctx->nvox = (long long)g.nx * g.ny * g.nz;
    ctx->clamp = o.clamp_nonneg ? 1 : 0;
    if (o.precision != 0 && o.precision != 1) {
        delete ctx;
        return fail(DEAM_ERR_ARG, "precision must be 0 (compensated) or 1 (plain FP32)");
    }
    ctx->fwd_mode = o.precision == 1 ? deam::FWD_DEAM_F32 : deam::FWD_DEAM;
    ctx->lambda = o.penalty_lambda;
    ctx->delta = o.penalty_lambda > 0.0 ? o.penalty_delta : 1.0;
    ctx->threshold = o.metal_threshold > 0.0 ? o.metal_threshold
                                             : 0.5 * std::min(g.dx, std::min(g.dy, g.nz > 1 ? g.dz : g.dx));
    ctx->slab = deam::context_slab(deam::pick_slab(g.nz, g.n_rows, g.dz, g.row_pitch, g.sid, g.sdd));
    ctx->n_slabs = (g.nz + ctx->slab - 1) / ctx->slab;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const long long ntiles = (long long)((g.n_channels + deam::kTileK - 1) / deam::kTileK) *
                             ((g.n_rows + deam::kTileR - 1) / deam::kTileR) *
                             ((g.n_views + deam::kTileV - 1) / deam::kTileV);
    ctx->n_fwd_blocks = (int)std::min<long long>(ntiles, (long long)sms * deam::forward_blocks_per_sm());

    // ---- geometry tables (double on the host, rounded once to float) ----
    const double X0 = g.cx - (g.nx - 1) / 2.0 * g.dx, Y0 = g.cy - (g.ny - 1) / 2.0 * g.dy,
                 Z0 = g.cz - (g.nz - 1) / 2.0 * g.dz;
    std::vector<float4> v4(g.n_views);
    std::vector<float> vz(g.n_views);
    for (int v = 0; v < g.n_views; ++v) {
        const double beta = g.start_angle + 2.0 * kPi * v / g.views_per_rotation;
        const double sx = g.sid * cos(beta), sy = g.sid * sin(beta);
        const double sz = g.z_start + g.feed * v / g.views_per_rotation;
        v4[v] = make_float4((float)((sx - X0) / g.dx), (float)((sy - Y0) / g.dy), (float)cos(beta), (float)sin(beta));
        vz[v] = (float)((sz - Z0) / g.dz);
    }
    std::vector<float2> ch(g.n_channels), rw(g.n_rows);
    for (int k = 0; k < g.n_channels; ++k) {
        const double gam = (k - (g.n_channels - 1) / 2.0 + g.channel_offset) * g.channel_pitch;
        ch[k] = make_float2((float)cos(gam), (float)sin(gam));
    }
    for (int r = 0; r < g.n_rows; ++r) {
        const double w = (r - (g.n_rows - 1) / 2.0 + g.row_offset) * g.row_pitch;
        rw[r] = make_float2((float)(w / g.dz), (float)sqrt(1.0 + (w / g.sdd) * (w / g.sdd)));
    }
    // per (slab, column tile) in the backprojector's block order
    const std::vector<int2> sv = deam::tile_view_ranges(g, ctx->slab, deam::kTileX, deam::kTileY);

    Geo& G = ctx->G;
    G.nx = g.nx; G.ny = g.ny; G.nz = g.nz; G.V = g.n_views; G.R = g.n_rows; G.K = g.n_channels;
    G.dx = (float)g.dx; G.dy = (float)g.dy;
    G.dx_sdd = (float)(g.dx / g.sdd); G.dy_sdd = (float)(g.dy / g.sdd);
    G.dx_dy = (float)(g.dx / g.dy); G.dy_dx = (float)(g.dy / g.dx);
    G.omega0 = (float)((0 - (g.n_rows - 1) / 2.0 + g.row_offset) * g.row_pitch / g.dz);
    G.domega = (float)(g.row_pitch / g.dz);
    G.chan_c0 = (float)((g.n_channels - 1) / 2.0 - g.channel_offset);
    G.inv_dgamma = (float)(1.0 / g.channel_pitch);
    G.vox_reach_mm = (float)(std::max(g.dx, g.dy) * 1.001);

    // ---- spectral tables ----
    Spec& S = ctx->S;
    const int nE = spectra->n_e;
    S.e_lo = nE;
    S.e_hi = 0;
    const double log2e = 1.4426950408889634;
    double mumax = 0.0;
    for (int e = 0; e < nE; ++e) {
        const double il = spectra->I0[e], ih = spectra->I0[nE + e];
        ctx->i0tot[0] += il;
        ctx->i0tot[1] += ih;
        const double m1 = basis->mu[e], m2 = basis->mu[nE + e];
        S.mu1l2[e] = (float)(m1 * log2e);
        S.mu2l2[e] = (float)(m2 * log2e);
        S.mu1[e] = (float)m1;
        S.mu2[e] = (float)m2;
        S.i0l[e] = (float)il;
        S.i0h[e] = (float)ih;
        if (il > 0.0 || ih > 0.0) {
            S.e_lo = std::min(S.e_lo, e);
            S.e_hi = std::max(S.e_hi, e + 1);
            mumax = std::max(mumax, m1 + m2);
        }
    }
    ctx->mumax = mumax;
    ctx->mu.assign(basis->mu, basis->mu + 2 * nE);
    ctx->i0.assign(spectra->I0, spectra->I0 + 2 * nE);
    if (spectra->energy_keV) ctx->energy.assign(spectra->energy_keV, spectra->energy_keV + nE);

    // ---- device buffers ----
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const size_t volx = (size_t)nx * (nz + 2) * (ny + 1), voly = (size_t)ny * (nz + 2) * (nx + 1);
    // allocations stop at the first failure (no further large requests once
    // the device has refused one)
    cudaError_t e = cudaSuccess;
#define DEAM_ALLOC(p, n)                        \
    do {                                        \
        if (e == cudaSuccess) e = dalloc(&(p), (n)); \
    } while (0)
    DEAM_ALLOC(ctx->view4, g.n_views);
    DEAM_ALLOC(ctx->view_z, g.n_views);
    DEAM_ALLOC(ctx->ip4, (size_t)g.n_views * g.n_channels);
    DEAM_ALLOC(ctx->ipL, (size_t)g.n_views * g.n_channels);
    DEAM_ALLOC(ctx->chan, g.n_channels);
    DEAM_ALLOC(ctx->row, g.n_rows);
    DEAM_ALLOC(ctx->slab_views, sv.size());
    DEAM_ALLOC(ctx->dt, (size_t)2 * ctx->nrays);
    DEAM_ALLOC(ctx->mask, (size_t)ctx->nrays);
    DEAM_ALLOC(ctx->payload, (size_t)ctx->nrays);
    DEAM_ALLOC(ctx->volX, volx);
    DEAM_ALLOC(ctx->volY, voly);
    DEAM_ALLOC(ctx->partial, (size_t)ctx->n_fwd_blocks);
    DEAM_ALLOC(ctx->scal, 4);
    DEAM_ALLOC(ctx->skipped, 1);
    DEAM_ALLOC(ctx->fault, 2);
    if (spectra->bowtie) DEAM_ALLOC(ctx->bowtie, g.n_channels);
    if (ctx->lambda > 0.0) DEAM_ALLOC(ctx->sums, (size_t)ctx->nvox);
#undef DEAM_ALLOC
    auto A = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_ctx(ctx);
        return fail(e == cudaErrorMemoryAllocation ? DEAM_ERR_OOM : DEAM_ERR_CUDA,
                    std::string("device allocation failed: ") + cudaGetErrorString(e));
    }
    G.view4 = ctx->view4;
    G.view_z = ctx->view_z;
    G.chan = ctx->chan;
    G.row = ctx->row;
    G.ip4 = ctx->ip4;
    G.ipL = ctx->ipL;
    G.fault = ctx->fault;
    A(cudaMemcpy(ctx->view4, v4.data(), sizeof(float4) * v4.size(), cudaMemcpyHostToDevice));
    A(cudaMemcpy(ctx->view_z, vz.data(), sizeof(float) * vz.size(), cudaMemcpyHostToDevice));
    A(cudaMemcpy(ctx->chan, ch.data(), sizeof(float2) * ch.size(), cudaMemcpyHostToDevice));
    A(cudaMemcpy(ctx->row, rw.data(), sizeof(float2) * rw.size(), cudaMemcpyHostToDevice));
    A(cudaMemcpy(ctx->slab_views, sv.data(), sizeof(int2) * sv.size(), cudaMemcpyHostToDevice));
    if (spectra->bowtie) {
        std::vector<float> bt(g.n_channels);
        for (int k = 0; k < g.n_channels; ++k) bt[k] = (float)spectra->bowtie[k];
        A(cudaMemcpy(ctx->bowtie, bt.data(), sizeof(float) * bt.size(), cudaMemcpyHostToDevice));
    }
    A(cudaMemset(ctx->mask, 0, (size_t)ctx->nrays));
    A(cudaMemset(ctx->fault, 0, 2 * sizeof(unsigned int)));
    A(deam::launch_inplane_table(G, ctx->ip4, ctx->ipL, 0));
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_ctx(ctx);
        return fail(DEAM_ERR_CUDA, std::string("table upload failed: ") + cudaGetErrorString(e));
    }

    // ---- normaliser Z = max_E(mu1+mu2) * max_y sum_x h(x,y) (projection of ones) ----
    if (o.Z > 0.0) {
        ctx->Z = o.Z;
    } else {
        cudaStream_t s = 0;
        int rc = build_layouts(ctx, nullptr, nullptr, 1, s);
        if (rc != DEAM_OK) {
            std::string m = g_err;
            free_ctx(ctx);
            return fail(rc, m);
        }
        deam::FwdArgs FA = fwd_args(ctx);
        e = deam::launch_forward(deam::FWD_MAX, ctx->G, ctx->S, FA, ctx->n_fwd_blocks, s);
        if (e == cudaSuccess) e = deam::launch_sum_partials(ctx->partial, ctx->n_fwd_blocks, ctx->scal, 1, s);
        double hmax = 0.0;
        if (e == cudaSuccess) e = cudaMemcpy(&hmax, ctx->scal, sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_ctx(ctx);
            return fail(DEAM_ERR_CUDA, std::string("normaliser projection failed: ") + cudaGetErrorString(e));
        }
        ctx->Z = mumax * hmax;
        if (!(ctx->Z > 0.0)) {
            free_ctx(ctx);
            return fail(DEAM_ERR_ARG, "normaliser Z is zero: no ray meets the volume or mu = 0");
        }
    }
    *out = ctx;
    return DEAM_OK;
}

int deam_destroy(deam_ctx* ctx) {
    if (!ctx) return DEAM_OK;
    if (ctx->batch_refs > 0) return fail(DEAM_ERR_STATE, "the context is part of a live batch: destroy the batch first");
    DeviceGuard dg(ctx->device);
    cudaDeviceSynchronize();
    free_ctx(ctx);
    return DEAM_OK;
}

int deam_info(deam_ctx* ctx, double* Z, long long* skipped_last) {
    if (!ctx) return fail(DEAM_ERR_ARG, "null context");
    if (Z) *Z = ctx->Z;
    if (skipped_last) *skipped_last = ctx->skipped_last;
    return DEAM_OK;
}

int deam_set_data(deam_ctx* ctx, const float* d, void* stream) {
    CHECK_CTX(ctx);
    if (!d) return fail(DEAM_ERR_ARG, "d must not be NULL");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = 2 * ctx->nrays;
    if (is_device_ptr(d)) {
        CK(deam::launch_clamp_copy(d, ctx->dt, n, s));
    } else {
        CK(cudaMemcpyAsync(ctx->dt, d, sizeof(float) * n, cudaMemcpyHostToDevice, s));
        CK(deam::launch_clamp_copy(ctx->dt, ctx->dt, n, s));
        CK(cudaStreamSynchronize(s));  // the caller's host buffer is released on return
    }
    ctx->has_data = true;
    return DEAM_OK;
}

int deam_set_metal_mask(deam_ctx* ctx, const void* m, int kind, void* stream) {
    CHECK_CTX(ctx);
    if (!m) return fail(DEAM_ERR_ARG, "m must not be NULL");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const bool dev = is_device_ptr(m);
    if (kind == DEAM_MASK_RAY || kind == DEAM_MASK_RAY_PER_SPECTRUM) {
        CK(cudaMemcpyAsync(ctx->mask, m, (size_t)ctx->nrays, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           s));
        CK(deam::launch_mask_bits(ctx->mask, ctx->nrays, kind == DEAM_MASK_RAY_PER_SPECTRUM, s));
        if (!dev) CK(cudaStreamSynchronize(s));  // the caller's host buffer is released on return
    } else if (kind == DEAM_MASK_VOXEL_IMAGE) {
        const float* M = (const float*)m;
        if (!dev) {
            // the payload buffer (16 B per ray) is free between calls: stage M there
            if ((long long)sizeof(float4) * ctx->nrays < (long long)sizeof(float) * ctx->nvox)
                return fail(DEAM_ERR_ARG, "host metal image larger than the staging buffer; pass device memory");
            CK(cudaMemcpyAsync(ctx->payload, M, sizeof(float) * ctx->nvox, cudaMemcpyHostToDevice, s));
            M = (const float*)ctx->payload;
        }
        int rc = build_layouts(ctx, nullptr, M, 0, s);
        if (rc != DEAM_OK) return rc;
        deam::FwdArgs A = fwd_args(ctx);
        A.mask_out = ctx->mask;
        A.threshold = (float)ctx->threshold;
        CK(deam::launch_forward(deam::FWD_MASK, ctx->G, ctx->S, A, ctx->n_fwd_blocks, s));
        if (!dev) CK(cudaStreamSynchronize(s));  // the caller's host buffer is released on return
    } else {
        return fail(DEAM_ERR_ARG, "unknown mask kind");
    }
    ctx->mask_set = true;
    return deam::finish_call(ctx, s);
}

int deam_get_metal_mask(deam_ctx* ctx, uint8_t* mask, void* stream) {
    CHECK_CTX(ctx);
    if (!mask) return fail(DEAM_ERR_ARG, "mask must not be NULL");
    DeviceGuard dg(ctx->device);
    NEED_DEVICE(mask, "mask");
    CK(cudaMemcpyAsync(mask, ctx->mask, (size_t)ctx->nrays, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return DEAM_OK;
}

int deam_forward(deam_ctx* ctx, const float* c, float* l, float* g, void* stream) {
    CHECK_CTX(ctx);
    if (!c || (!l && !g)) return fail(DEAM_ERR_ARG, "need c and at least one of l, g");
    DeviceGuard dg(ctx->device);
    NEED_DEVICE(c, "c");
    NEED_DEVICE(l, "l");
    NEED_DEVICE(g, "g");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = build_layouts(ctx, (const float2*)c, nullptr, 0, s);
    if (rc != DEAM_OK) return rc;
    deam::FwdArgs A = fwd_args(ctx);
    A.l_out = (float2*)l;
    A.g_out = g;
    CK(deam::launch_forward(g ? deam::FWD_LINE_G : deam::FWD_LINE, ctx->G, ctx->S, A, ctx->n_fwd_blocks, s));
    return deam::finish_call(ctx, s);
}

int deam_backproject(deam_ctx* ctx, const float* y, float* img, void* stream) {
    CHECK_CTX(ctx);
    if (!y || !img) return fail(DEAM_ERR_ARG, "y and img must not be NULL");
    DeviceGuard dg(ctx->device);
    NEED_DEVICE(y, "y");
    NEED_DEVICE(img, "img");
    deam::BwdArgs B{};
    B.rays2 = (const float2*)y;
    B.img = (float2*)img;
    B.slab_views = ctx->slab_views;
    CK(deam::launch_backward(deam::BWD_ADJOINT, ctx->slab, ctx->G, B, (cudaStream_t)stream));
    return deam::finish_call(ctx, (cudaStream_t)stream);
}

// fold = 1: the payload in the backprojector's internal form (times the row
// length factor); 0: as defined in deam.h (deam_ray_terms).
static int ray_terms(deam_ctx* ctx, const float2* c, float4* payload, double* F, double* F_dev, cudaStream_t s,
                     int fold) {
    int rc = build_layouts(ctx, c, nullptr, 0, s);
    if (rc != DEAM_OK) return rc;
    deam::FwdArgs A = fwd_args(ctx);
    A.dt = ctx->dt;
    A.mask = ctx->mask_set ? ctx->mask : nullptr;
    A.payload = payload;
    A.fold_rowfac = fold;
    CK(deam::launch_forward(ctx->fwd_mode, ctx->G, ctx->S, A, ctx->n_fwd_blocks, s));
    CK(deam::launch_sum_partials(ctx->partial, ctx->n_fwd_blocks, F_dev, 0, s));
    if (F) {
        CK(cudaMemcpyAsync(F, F_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return deam::finish_call(ctx, s);
}

int deam_ray_terms(deam_ctx* ctx, const float* c, float* payload, double* F, void* stream) {
    CHECK_CTX(ctx);
    if (!c || !payload) return fail(DEAM_ERR_ARG, "c and payload must not be NULL");
    if (!ctx->has_data) return fail(DEAM_ERR_STATE, "deam_set_data has not been called");
    DeviceGuard dg(ctx->device);
    NEED_DEVICE(c, "c");
    NEED_DEVICE(payload, "payload");
    return ray_terms(ctx, (const float2*)c, (float4*)payload, F, ctx->scal, (cudaStream_t)stream, 0);
}

int deam_objective(deam_ctx* ctx, const float* c, double* out, void* stream) {
    CHECK_CTX(ctx);
    if (!c || !out) return fail(DEAM_ERR_ARG, "c and out must not be NULL");
    if (!ctx->has_data) return fail(DEAM_ERR_STATE, "deam_set_data has not been called");
    DeviceGuard dg(ctx->device);
    NEED_DEVICE(c, "c");
    int rc = ray_terms(ctx, (const float2*)c, ctx->payload, out, ctx->scal, (cudaStream_t)stream, 0);
    if (rc == DEAM_OK && !isfinite(*out)) return fail(DEAM_ERR_NUMERIC, "objective is not finite");
    return rc;
}

int deam_iterate(deam_ctx* ctx, float* c, int n_iter, double* hist, void* stream) {
    CHECK_CTX(ctx);
    if (!c) return fail(DEAM_ERR_ARG, "c must not be NULL");
    if (n_iter < 0) return fail(DEAM_ERR_ARG, "n_iter must be >= 0");
    if (!ctx->has_data) return fail(DEAM_ERR_STATE, "deam_set_data has not been called");
    if (n_iter == 0) return DEAM_OK;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    float2* cd = (float2*)c;
    const bool host = !is_device_ptr(c);
    if (host) {
        if (!ctx->c_stage) CK(dalloc(&ctx->c_stage, (size_t)ctx->nvox));
        CK(cudaMemcpyAsync(ctx->c_stage, c, sizeof(float2) * ctx->nvox, cudaMemcpyHostToDevice, s));
        cd = ctx->c_stage;
    }
    if (ctx->hist_cap < n_iter) {
        if (ctx->hist) CK(cudaFree(ctx->hist));
        ctx->hist = nullptr;
        ctx->hist_cap = 0;
        CK(dalloc(&ctx->hist, (size_t)n_iter));
        ctx->hist_cap = n_iter;
    }
    deam::BwdArgs B{};
    B.payload = ctx->payload;
    B.img = cd;
    B.slab_views = ctx->slab_views;
    B.invZ = 1.0 / ctx->Z;
    B.clamp_nonneg = ctx->clamp;
    B.skipped = ctx->skipped;
    deam::set_penalty_args(ctx, B);
    std::vector<cudaEvent_t> ev;
    if (ctx->prof) {
        ev.resize((size_t)5 * n_iter);
        for (auto& x : ev) CK(cudaEventCreate(&x));
    }
    deam::FwdArgs A = fwd_args(ctx);
    A.dt = ctx->dt;
    A.mask = ctx->mask_set ? ctx->mask : nullptr;
    A.payload = ctx->payload;
    A.fold_rowfac = 1;
    NvtxRange iter_range("deam_iterate");
    for (int it = 0; it < n_iter; ++it) {
        cudaEvent_t* e = ctx->prof ? &ev[(size_t)5 * it] : nullptr;
        if (e) CK(cudaEventRecord(e[0], s));
        {
            NvtxRange r("deam.layout");
            int rc = build_layouts(ctx, cd, nullptr, 0, s);
            if (rc != DEAM_OK) return rc;
        }
        if (e) CK(cudaEventRecord(e[1], s));
        {
            NvtxRange r("deam.forward");  // Joseph projection + spectral sums + substitution + p-step + F partials
            CK(deam::launch_forward(ctx->fwd_mode, ctx->G, ctx->S, A, ctx->n_fwd_blocks, s));
        }
        if (e) CK(cudaEventRecord(e[2], s));
        {
            NvtxRange r("deam.objective");
            CK(deam::launch_sum_partials(ctx->partial, ctx->n_fwd_blocks, ctx->hist + it, 0, s));
            CK(cudaMemsetAsync(ctx->skipped, 0, sizeof(unsigned long long), s));
        }
        if (e) CK(cudaEventRecord(e[3], s));
        {
            NvtxRange r("deam.backproject");  // gather backprojection + c-step
            CK(deam::launch_backward(deam::BWD_UPDATE, ctx->slab, ctx->G, B, s));
            if (B.sums) CK(deam::launch_reg_update(ctx->G, B, s));
        }
        if (e) CK(cudaEventRecord(e[4], s));
    }
    unsigned long long sk = 0;
    CK(cudaMemcpyAsync(&sk, ctx->skipped, sizeof(sk), cudaMemcpyDeviceToHost, s));
    std::vector<double> h(n_iter);
    CK(cudaMemcpyAsync(h.data(), ctx->hist, sizeof(double) * n_iter, cudaMemcpyDeviceToHost, s));
    if (host) CK(cudaMemcpyAsync(c, ctx->c_stage, sizeof(float2) * ctx->nvox, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    {
        const int rc = deam::finish_call(ctx, s);
        if (rc != DEAM_OK) return rc;
    }
    ctx->skipped_last = (long long)sk;
    if (ctx->prof) {
        const int nl[4] = {2, 1, 1, 1};
        for (int it = 0; it < n_iter; ++it)
            for (int j = 0; j < 4; ++j) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, ev[(size_t)5 * it + j], ev[(size_t)5 * it + j + 1]));
                ctx->prof_ms[j] += ms;
                ctx->prof_n[j] += nl[j];
            }
        for (auto& x : ev) cudaEventDestroy(x);
    }
    if (hist) memcpy(hist, h.data(), sizeof(double) * n_iter);
    for (double v : h)
        if (!isfinite(v)) return fail(DEAM_ERR_NUMERIC, "objective became non-finite");
    return DEAM_OK;
}

int deam_backprojected_sums(deam_ctx* ctx, const float* c, float* sums, double* F, double* Z, void* stream) {
    CHECK_CTX(ctx);
    if (!c || !sums) return fail(DEAM_ERR_ARG, "c and sums must not be NULL");
    if (!ctx->has_data) return fail(DEAM_ERR_STATE, "deam_set_data has not been called");
    DeviceGuard dg(ctx->device);
    NEED_DEVICE(c, "c");
    NEED_DEVICE(sums, "sums");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ray_terms(ctx, (const float2*)c, ctx->payload, nullptr, ctx->scal, s, 1);
    if (rc != DEAM_OK) return rc;
    deam::BwdArgs B{};
    B.payload = ctx->payload;
    B.slab_views = ctx->slab_views;
    B.sums = (float4*)sums;  // the c-step's backprojection, stopped before the update
    CK(deam::launch_backward(deam::BWD_UPDATE, ctx->slab, ctx->G, B, s));
    rc = deam::finish_call(ctx, s);
    if (rc != DEAM_OK) return rc;
    if (Z) *Z = ctx->Z;
    if (F) {
        CK(cudaMemcpyAsync(F, ctx->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!isfinite(*F)) return fail(DEAM_ERR_NUMERIC, "objective is not finite");
    }
    return DEAM_OK;
}

int deam_gradient(deam_ctx* ctx, const float* c, float* grad, double* F, void* stream) {
    CHECK_CTX(ctx);
    if (!c || !grad) return fail(DEAM_ERR_ARG, "c and grad must not be NULL");
    if (!ctx->has_data) return fail(DEAM_ERR_STATE, "deam_set_data has not been called");
    DeviceGuard dg(ctx->device);
    NEED_DEVICE(c, "c");
    NEED_DEVICE(grad, "grad");
    cudaStream_t s = (cudaStream_t)stream;
    // per-ray terms recomputed from c (nothing per energy bin is stored), then
    // the gather backprojection of D = sum_j (r_j - 1) S_ij gives b^ - b~
    int rc = ray_terms(ctx, (const float2*)c, ctx->payload, nullptr, ctx->scal, s, 1);
    if (rc != DEAM_OK) return rc;
    deam::BwdArgs B{};
    B.payload = ctx->payload;
    B.img = (float2*)grad;
    B.slab_views = ctx->slab_views;
    CK(deam::launch_backward(deam::BWD_GRADIENT, ctx->slab, ctx->G, B, s));
    rc = deam::finish_call(ctx, s);
    if (rc != DEAM_OK) return rc;
    if (F) {
        CK(cudaMemcpyAsync(F, ctx->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!isfinite(*F)) return fail(DEAM_ERR_NUMERIC, "objective is not finite");
    }
    return DEAM_OK;
}

int deam_penalty(deam_ctx* ctx, const float* c, double* R, void* stream) {
    CHECK_CTX(ctx);
    if (!c || !R) return fail(DEAM_ERR_ARG, "c and R must not be NULL");
    DeviceGuard dg(ctx->device);
    NEED_DEVICE(c, "c");
    cudaStream_t s = (cudaStream_t)stream;
    const deam_geometry& g = ctx->geo;
    CK(deam::launch_penalty((const float2*)c, g.nx, g.ny, g.nz, (float)g.dx, (float)g.dy, (float)g.dz,
                            (float)ctx->lambda, (float)ctx->delta, ctx->partial, ctx->n_fwd_blocks, s));
    CK(deam::launch_sum_partials(ctx->partial, ctx->n_fwd_blocks, ctx->scal + 2, 0, s));
    CK(cudaMemcpyAsync(R, ctx->scal + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return DEAM_OK;
}

int deam_basis_images(deam_ctx* ctx, const float* c, const double* coef, int n, float* out, void* stream) {
    CHECK_CTX(ctx);
    if (!c || !coef || !out || n < 1 || n > 256) return fail(DEAM_ERR_ARG, "need c, out and 1..256 coefficient pairs");
    for (int e = 0; e < 2 * n; ++e)
        if (!isfinite(coef[e])) return fail(DEAM_ERR_ARG, "coefficients must be finite");
    DeviceGuard dg(ctx->device);
    NEED_DEVICE(c, "c");
    NEED_DEVICE(out, "out");
    cudaStream_t s = (cudaStream_t)stream;
    if (!ctx->coef) CK(dalloc(&ctx->coef, 256));
    std::vector<float2> ab(n);
    for (int e = 0; e < n; ++e) ab[e] = make_float2((float)coef[2 * e], (float)coef[2 * e + 1]);
    CK(cudaMemcpyAsync(ctx->coef, ab.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, s));
    CK(deam::launch_combine((const float2*)c, ctx->nvox, ctx->coef, n, out, s));
    CK(cudaStreamSynchronize(s));  // the host coefficient buffer is released on return
    return DEAM_OK;
}

// mu_i(E) of the context's tables at energy E: linear interpolation of
// ln mu_i between the bin centres, the end values beyond them.
static double mu_at(const deam_ctx* ctx, int i, double E) {
    const std::vector<double>& x = ctx->energy;
    const int n = (int)x.size();
    auto lg = [&](int e) { return log(std::max(ctx->mu[(size_t)i * n + e], 1e-300)); };
    if (E <= x[0]) return exp(lg(0));
    if (E >= x[n - 1]) return exp(lg(n - 1));
    int e = (int)(std::upper_bound(x.begin(), x.end(), E) - x.begin()) - 1;
    const double t = (E - x[e]) / (x[e + 1] - x[e]);
    return exp(lg(e) + t * (lg(e + 1) - lg(e)));
}

int deam_vmi(deam_ctx* ctx, const float* c, const double* energies, int n, float* out, void* stream) {
    CHECK_CTX(ctx);
    if (!energies || n < 1 || n > 256) return fail(DEAM_ERR_ARG, "need 1..256 energies");
    if (ctx->energy.empty()) return fail(DEAM_ERR_STATE, "the context was created without bin energies");
    for (size_t e = 1; e < ctx->energy.size(); ++e)
        if (!(ctx->energy[e] > ctx->energy[e - 1])) return fail(DEAM_ERR_STATE, "bin energies must increase");
    std::vector<double> coef(2 * (size_t)n);
    for (int e = 0; e < n; ++e) {
        if (!isfinite(energies[e])) return fail(DEAM_ERR_ARG, "energies must be finite");
        coef[2 * e] = mu_at(ctx, 0, energies[e]);
        coef[2 * e + 1] = mu_at(ctx, 1, energies[e]);
    }
    return deam_basis_images(ctx, c, coef.data(), n, out, stream);
}

int deam_kvp_images(deam_ctx* ctx, const float* c, float* out, void* stream) {
    CHECK_CTX(ctx);
    const size_t nE = ctx->i0.size() / 2;
    double coef[4] = {0, 0, 0, 0};
    for (int j = 0; j < 2; ++j) {
        double tot = 0.0;
        for (size_t e = 0; e < nE; ++e) tot += ctx->i0[j * nE + e];
        if (!(tot > 0.0)) return fail(DEAM_ERR_STATE, "an empty spectrum has no weighted image");
        for (size_t e = 0; e < nE; ++e) {
            const double w = ctx->i0[j * nE + e] / tot;
            coef[2 * j] += w * ctx->mu[e];
            coef[2 * j + 1] += w * ctx->mu[nE + e];
        }
    }
    return deam_basis_images(ctx, c, coef, 2, out, stream);
}

int deam_count_samples(deam_ctx* ctx, long long* n, void* stream) {
    CHECK_CTX(ctx);
    if (!n) return fail(DEAM_ERR_ARG, "n must not be NULL");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    deam::FwdArgs A = fwd_args(ctx);
    CK(deam::launch_forward(deam::FWD_COUNT, ctx->G, ctx->S, A, ctx->n_fwd_blocks, s));
    CK(deam::launch_sum_partials(ctx->partial, ctx->n_fwd_blocks, ctx->scal + 1, 0, s));
    double v = 0.0;
    CK(cudaMemcpyAsync(&v, ctx->scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *n = (long long)llround(v);
    return DEAM_OK;
}

int deam_bounds_checked(void) {
#ifdef DEAM_BOUNDS_CHECK
    return 1;
#else
    return 0;
#endif
}

int deam_bounds_inject(deam_ctx* ctx, void* stream) {
    CHECK_CTX(ctx);
#ifdef DEAM_BOUNDS_CHECK
    DeviceGuard dg(ctx->device);
    const unsigned int w[2] = {deam::SITE_INJECTED, 0};
    CK(cudaMemcpyAsync(ctx->fault, w, sizeof(w), cudaMemcpyHostToDevice, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return DEAM_OK;
#else
    (void)stream;
    return fail(DEAM_ERR_STATE, "not a bounds-checked build (compile with -DDEAM_BOUNDS_CHECK)");
#endif
}

int deam_l1_bandwidth(double* bytes_per_s, void* stream) {
    if (!bytes_per_s) return fail(DEAM_ERR_ARG, "bytes_per_s must not be NULL");
    cudaError_t e = deam::l1_probe(bytes_per_s, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(DEAM_ERR_CUDA, std::string("l1 probe: ") + cudaGetErrorString(e));
    return DEAM_OK;
}

int deam_profile(deam_ctx* ctx, int enable) {
    CHECK_CTX(ctx);
    ctx->prof = enable != 0;
    return DEAM_OK;
}

int deam_kernel_times(deam_ctx* ctx, double* ms, long long* launches, int reset) {
    if (!ctx) return fail(DEAM_ERR_ARG, "null context");
    for (int j = 0; j < 4; ++j) {
        if (ms) ms[j] = ctx->prof_ms[j];
        if (launches) launches[j] = ctx->prof_n[j];
        if (reset) {
            ctx->prof_ms[j] = 0.0;
            ctx->prof_n[j] = 0;
        }
    }
    return DEAM_OK;
}

}  // extern "C"
