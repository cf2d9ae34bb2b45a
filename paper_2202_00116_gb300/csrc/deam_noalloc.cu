// deam_objective_noalloc: the MAR-DEAM objective F(c) for callers that cannot
// allocate device memory.
//
// Who cannot allocate: code that runs where cudaMalloc is forbidden or harmful --
// inside a region whose device memory is owned by someone else (a framework's
// caching allocator or a fixed arena that must not be bypassed), in a
// latency-bound loop where cudaMalloc/cudaFree would synchronise the device, or
// on a process that has no spare device memory left for a context's buffers.
// Such a caller owns its inputs and outputs but cannot create a deam_ctx, whose
// buffers are allocated by deam_init.
//
// This entry point therefore takes only caller-owned pointers and keeps its one
// piece of scratch -- the FP64 objective partial of each 128-ray block -- in a
// file-scope static device array of fixed size.  Every GPU that loads the
// library holds that array until the process exits.  All calls share it, so
// calls that overlap on the GPU (two streams, or two host threads) race on it;
// serialise them.  It keeps the last call's contents; nothing in it has to
// start at zero, because each call writes every partial it later reads.
#include <math.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "deam.h"
#include "deam_epilogue.cuh"
#include "deam_internal.h"

namespace {

constexpr int kThreads = 128;                         // rays per block = rays per partial
constexpr long long kMaxPartials = 1LL << 20;         // 8 MiB of FP64 partials
constexpr long long kMaxRays = kMaxPartials * kThreads;  // 134,217,728 rays
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kMaxPartials];

// Device address of g_noalloc_partials per device.  In host code the array's
// name is only a host-side stand-in; the address must come from
// cudaGetSymbolAddress with the device current.
std::mutex g_mu;
double* g_scratch[kMaxDevices] = {};

cudaError_t scratch_of(int dev, double** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        double* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return cudaSuccess;
}

int err(int code, const char* m) { return deam::set_error(code, m); }

constexpr int kMaxBowtie = 1024;
struct Bowtie {
    int on;
    float b[kMaxBowtie];
};

// Scalar geometry of the scan (no device tables: computed per ray).
struct ScanGeo {
    int nx, ny, nz, V, R, K, vpr;
    double start, sid, sdd, feed, z_start, X0, Y0, Z0, dx, dy, dz;
    double ch_c, ch_pitch, row_c, row_pitch;
};

// Variant of the forward kernel's DEAM mode: the same Joseph sampling
// (ray_inplane / row_fz) but gathering the four taps straight from the caller's
// image [nz][ny][nx] with bounds tests instead of the context's paired layouts,
// the per-view/channel/row terms computed per ray in double and rounded once (as
// the context's tables are), only the objective in the epilogue, and the
// per-block FP64 partials written to the static scratch.
__global__ void __launch_bounds__(kThreads) objective_image_kernel(const ScanGeo SG, const deam::Geo G,
                                                                   const deam::Spec S, const float2* __restrict__ c,
                                                                   const float* __restrict__ d,
                                                                   const uint8_t* __restrict__ mask,
                                                                   const Bowtie BT, double* __restrict__ partials) {
    const long long nrays = (long long)SG.V * SG.R * SG.K;
    const long long y = (long long)blockIdx.x * kThreads + threadIdx.x;
    double f = 0.0;
    if (y < nrays) {
        const int k = (int)(y % SG.K);
        const long long vr = y / SG.K;
        const int r = (int)(vr % SG.R);
        const int v = (int)(vr / SG.R);
        const double beta = SG.start + 2.0 * 3.14159265358979323846 * v / SG.vpr;
        double sb, cb;
        sincos(beta, &sb, &cb);
        const double gam = (k - SG.ch_c) * SG.ch_pitch;
        double sg, cg;
        sincos(gam, &sg, &cg);
        const double w = (r - SG.row_c) * SG.row_pitch;
        const float4 vw = make_float4((float)((SG.sid * cb - SG.X0) / SG.dx), (float)((SG.sid * sb - SG.Y0) / SG.dy),
                                      (float)cb, (float)sb);
        const float sz = (float)((SG.z_start + SG.feed * v / SG.vpr - SG.Z0) / SG.dz);
        const float omega = deam::row_omega(G, r);
        const float lz = (float)sqrt(1.0 + (w / SG.sdd) * (w / SG.sdd));
        const deam::InPlane ip = deam::ray_inplane(G, vw, make_float2((float)cg, (float)sg));
        const int np = ip.axis ? SG.ny : SG.nx;
        const int nq = ip.axis ? SG.nx : SG.ny;
        float s1 = 0.f, s2 = 0.f;
        for (int p = 0; p < np; ++p) {
            const float pf = (float)p;
            const float fq = __fmaf_rn(pf, ip.bq, ip.aq);
            const float fz = deam::row_fz(sz, omega, deam::ray_t(ip, pf));
            if (!(fq >= -1.f && fq < (float)nq && fz >= -1.f && fz < (float)SG.nz)) continue;
            const float jqf = floorf(fq), jzf = floorf(fz);
            const float wq = fq - jqf, wz = fz - jzf;
            const int jq = (int)jqf, jz = (int)jzf;
            float2 t[2][2];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const int q = jq + b, z = jz + a;
                    t[a][b] = make_float2(0.f, 0.f);
                    if (q >= 0 && q < nq && z >= 0 && z < SG.nz) {
                        const int ix = ip.axis ? q : p, iy = ip.axis ? p : q;
                        t[a][b] = c[((long long)z * SG.ny + iy) * SG.nx + ix];
                    }
                }
            const float a1 = fmaf(wq, t[0][1].x - t[0][0].x, t[0][0].x), b1 = fmaf(wq, t[1][1].x - t[1][0].x, t[1][0].x);
            const float a2 = fmaf(wq, t[0][1].y - t[0][0].y, t[0][0].y), b2 = fmaf(wq, t[1][1].y - t[1][0].y, t[1][0].y);
            s1 += fmaf(wz, b1 - a1, a1);
            s2 += fmaf(wz, b2 - a2, a2);
        }
        const float L = __fmul_rn(ip.Lxy, lz);
        const float l1 = s1 * L, l2 = s2 * L;
        // bit j of the mask: the ray is on the metal trace of spectrum j, whose
        // data term is then left out (Eq. 11: p = q there)
        const unsigned mk = mask ? (unsigned)mask[y] : 0u;
        if ((mk & 3u) != 3u) {
            float gl, gh, u1, u2, u3, u4;
            deam::spectral_sums<false>(S, l1, l2, gl, gh, u1, u2, u3, u4);
            const float bk = BT.on ? BT.b[k] : 1.f;
            gl *= bk;
            gh *= bk;
            float ff = 0.f;
            if (!(mk & 1u)) {
                const float dl = fmaxf(d[y], 0.f);
                if (gl > 0.f) ff = fmaf(gl, deam::idiv_phi((dl - gl) / gl), ff);
                else if (dl > 0.f) ff = INFINITY;
            }
            if (!(mk & 2u)) {
                const float dh = fmaxf(d[nrays + y], 0.f);
                if (gh > 0.f) ff = fmaf(gh, deam::idiv_phi((dh - gh) / gh), ff);
                else if (dh > 0.f) ff = INFINITY;
            }
            f = (double)ff;
        }
    }
    const double b = deam::block_reduce<kThreads, double>(f, false);
    if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

// Device (or managed) memory: a host buffer here would fault the kernel.
bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int deam_objective_noalloc(const deam_geometry* geom, const deam_spectra* spectra,
                                      const deam_basis* basis, const float* c, const float* d,
                                      const uint8_t* mask, double* F, void* stream) {
    if (!geom || !spectra || !basis || !c || !d || !F)
        return err(DEAM_ERR_ARG, "deam_objective_noalloc: geometry, spectra, basis, c, d and F must not be NULL");
    if (!on_device(c) || !on_device(d) || !on_device(F) || (mask && !on_device(mask)))
        return err(DEAM_ERR_ARG, "deam_objective_noalloc: c, d, mask and F must be device memory");
    const deam_geometry& g = *geom;
    // the same host-side checks as deam_init (geometry inside the source circle,
    // finite values, table sizes): a scan the context refuses is refused here too
    const std::string why = deam::validate_scan(geom, spectra, basis);
    if (!why.empty()) return err(DEAM_ERR_ARG, ("deam_objective_noalloc: " + why).c_str());
    const long long nrays = (long long)g.n_views * g.n_rows * g.n_channels;
    if (nrays > kMaxRays)
        return err(DEAM_ERR_ARG, "deam_objective_noalloc: more than 134217728 rays (the static scratch holds "
                                 "one FP64 partial per 128 rays, 8 MiB)");
    if ((double)g.nx * g.ny * g.nz > 2147483647.0) return err(DEAM_ERR_ARG, "deam_objective_noalloc: volume too large");
    if (spectra->n_e < 1 || spectra->n_e > deam::kMaxE || basis->n_e != spectra->n_e || !spectra->I0 || !basis->mu)
        return err(DEAM_ERR_ARG, "deam_objective_noalloc: need 1 <= n_e <= 256 bins, equal in spectra and basis");
    Bowtie BT;
    BT.on = spectra->bowtie != nullptr;
    if (BT.on) {
        if (g.n_channels > kMaxBowtie)
            return err(DEAM_ERR_ARG, "deam_objective_noalloc: a bowtie is limited to 1024 channels");
        for (int k = 0; k < g.n_channels; ++k) {
            if (!finite_pos(spectra->bowtie[k]))
                return err(DEAM_ERR_ARG, "deam_objective_noalloc: bowtie factors must be finite and > 0");
            BT.b[k] = (float)spectra->bowtie[k];
        }
    }

    // spectral tables as kernel parameters (host struct: no allocation)
    deam::Spec S;
    const int nE = spectra->n_e;
    S.e_lo = nE;
    S.e_hi = 0;
    const double log2e = 1.4426950408889634;
    for (int e = 0; e < nE; ++e) {
        const double il = spectra->I0[e], ih = spectra->I0[nE + e], m1 = basis->mu[e], m2 = basis->mu[nE + e];
        if (!(isfinite(il) && il >= 0.0 && isfinite(ih) && ih >= 0.0 && isfinite(m1) && m1 >= 0.0 && isfinite(m2) &&
              m2 >= 0.0))
            return err(DEAM_ERR_ARG, "deam_objective_noalloc: I0 and mu must be finite and >= 0");
        S.mu1l2[e] = (float)(m1 * log2e);
        S.mu2l2[e] = (float)(m2 * log2e);
        S.mu1[e] = (float)m1;
        S.mu2[e] = (float)m2;
        S.i0l[e] = (float)il;
        S.i0h[e] = (float)ih;
        if (il > 0.0 || ih > 0.0) {
            if (e < S.e_lo) S.e_lo = e;
            S.e_hi = e + 1;
        }
    }
    if (S.e_hi == 0) return err(DEAM_ERR_ARG, "deam_objective_noalloc: both spectra are empty");

    ScanGeo SG;
    SG.nx = g.nx; SG.ny = g.ny; SG.nz = g.nz; SG.V = g.n_views; SG.R = g.n_rows; SG.K = g.n_channels;
    SG.vpr = g.views_per_rotation;
    SG.start = g.start_angle; SG.sid = g.sid; SG.sdd = g.sdd; SG.feed = g.feed; SG.z_start = g.z_start;
    SG.X0 = g.cx - (g.nx - 1) / 2.0 * g.dx;
    SG.Y0 = g.cy - (g.ny - 1) / 2.0 * g.dy;
    SG.Z0 = g.cz - (g.nz - 1) / 2.0 * g.dz;
    SG.dx = g.dx; SG.dy = g.dy; SG.dz = g.dz;
    SG.ch_c = (g.n_channels - 1) / 2.0 - g.channel_offset;
    SG.ch_pitch = g.channel_pitch;
    SG.row_c = (g.n_rows - 1) / 2.0 - g.row_offset;
    SG.row_pitch = g.row_pitch;
    deam::Geo G{};
    G.nx = g.nx; G.ny = g.ny; G.nz = g.nz; G.V = g.n_views; G.R = g.n_rows; G.K = g.n_channels;
    G.dx = (float)g.dx; G.dy = (float)g.dy;
    G.dx_sdd = (float)(g.dx / g.sdd); G.dy_sdd = (float)(g.dy / g.sdd);
    G.dx_dy = (float)(g.dx / g.dy); G.dy_dx = (float)(g.dy / g.dx);
    G.omega0 = (float)((0 - (g.n_rows - 1) / 2.0 + g.row_offset) * g.row_pitch / g.dz);
    G.domega = (float)(g.row_pitch / g.dz);

    // set-up on this device (first call only): the scratch's device address
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(DEAM_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(DEAM_ERR_ARG, "deam_objective_noalloc: device ordinal >= 64");
    double* scratch = nullptr;
    e = scratch_of(dev, &scratch);
    if (e != cudaSuccess) return err(DEAM_ERR_CUDA, cudaGetErrorString(e));

    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)((nrays + kThreads - 1) / kThreads);
    objective_image_kernel<<<blocks, kThreads, 0, s>>>(SG, G, S, (const float2*)c, d, mask, BT, scratch);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = deam::launch_sum_partials(scratch, blocks, F, 0, s);
    if (e != cudaSuccess) return err(DEAM_ERR_CUDA, cudaGetErrorString(e));
    return DEAM_OK;
}
