// Internal declarations shared by the kernels (deam_kernels.cu) and the C ABI
// (deam_api.cu) of the sm_103a MAR-DEAM library.  Not installed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "deam.h"

namespace deam {

constexpr int kMaxE = 256;        // energy bins carried in the kernel-parameter tables
constexpr int kTileK = 32;        // forward ray tile: channels (one warp) ...
constexpr int kTileR = 4;         // ... x rows ...
constexpr int kTileV = 2;         // ... x views
constexpr int kFwdThreads = kTileK * kTileR * kTileV;  // rays per forward block (256)
constexpr int kTileX = 16;        // backprojector column tile (x)
constexpr int kTileY = 8;         // backprojector column tile (y)

// Geometry in voxel-index units, as read by both projector directions.  Every
// per-ray quantity is derived from these tables by ray_inplane()/row terms with
// explicitly rounded FP32 operations, so the forward and the gather-backward
// kernels compute bit-identical sample positions and weights.
struct Geo {
    int nx, ny, nz, V, R, K;
    float dx, dy;            // voxel edge lengths (mm)
    float dx_sdd, dy_sdd;    // dx / sdd, dy / sdd
    float dx_dy, dy_dx;      // dx / dy, dy / dx
    const float4* view4;     // [V] (sigma_x, sigma_y, cos beta, sin beta); sigma = source in index units
    const float* view_z;     // [V] sigma_z = (s_z - Z0) / dz
    const float2* chan;      // [K] (cos gamma_k, sin gamma_k)
    const float2* row;       // [R] (w_r / dz, sqrt(1 + (w_r/sdd)^2)): .y is the row length factor
    const float4* ip4;       // [V][K] (aq, bq, tau0, kappa) of ray_inplane, built once by build_inplane_table
    const float* ipL;        // [V][K] Lxy, negated for y-dominant rays
    float omega0, domega;    // omega_r = omega0 + r domega (row_omega)
    float chan_c0, inv_dgamma;  // channel coordinate = gamma / dgamma + chan_c0
    float vox_reach_mm;      // max(dx, dy): reach of a voxel's bilinear footprint in-plane
    unsigned int* fault;     // [2] bounds-checked builds: first failing site and index (else unused)
};

// Bounds-checked builds (-DDEAM_BOUNDS_CHECK): every guarded access tests its
// index first; a failing test records (site, index) in the context's fault
// words -- the first one only -- and the access is skipped, so the kernel
// finishes and the entry point reports DEAM_ERR_ARG on return.  Never traps.
enum BoundsSite : unsigned {
    SITE_FWD_LAYOUT = 1,   // forward: paired-layout gather
    SITE_FWD_RAY = 2,      // forward: per-ray data (d~, mask, payload, outputs)
    SITE_BWD_RAY = 3,      // backprojection: ray data / payload gather
    SITE_BWD_TABLE = 4,    // backprojection: in-plane ray table
    SITE_BWD_IMAGE = 5,    // backprojection: image / sums
    SITE_INJECTED = 99     // written from the host by deam_bounds_inject
};
#ifdef DEAM_BOUNDS_CHECK
__device__ __forceinline__ bool in_bounds(unsigned int* fault, bool ok, unsigned site, long long idx) {
    if (!ok && fault && atomicCAS(fault, 0u, site) == 0u) fault[1] = (unsigned)(idx < 0 ? 0xffffffffu : idx);
    return ok;
}
#define DEAM_IN_BOUNDS(G, cond, site, idx) ::deam::in_bounds((G).fault, (cond), (site), (long long)(idx))
#else
#define DEAM_IN_BOUNDS(G, cond, site, idx) true
#endif

// Spectral model tables (kernel parameters: they live in the constant bank).
struct Spec {
    int e_lo, e_hi;                  // active bins [e_lo, e_hi)
    float mu1l2[kMaxE], mu2l2[kMaxE];  // mu_i(E) * log2(e), 1/mm
    float mu1[kMaxE], mu2[kMaxE];      // mu_i(E), 1/mm
    float i0l[kMaxE], i0h[kMaxE];      // I0_j(E), counts
};

struct InPlane {
    int axis;      // 0: x-dominant (planes ix), 1: y-dominant (planes iy)
    float aq, bq;  // fq(p) = aq + p bq: intercept with plane p on the other transaxial axis (index units)
    float tau0, kappa;  // ray parameter t(p) = tau0 + p kappa (fraction of u)
    float Lxy;     // (plane spacing) / |d_dominant|; times the row factor gives Joseph's L
};

// In-plane ray parameters of (view, channel).  Explicitly rounded operations
// (no contraction freedom) make the result identical wherever it is inlined.
__device__ __forceinline__ InPlane ray_inplane(const Geo& G, float4 vw, float2 ch) {
    // d_k = -(cos(beta + gamma), sin(beta + gamma)) by the angle-sum identities
    const float dxk = __fmaf_rn(vw.w, ch.y, -__fmul_rn(vw.z, ch.x));
    const float dyk = -__fmaf_rn(vw.w, ch.x, __fmul_rn(vw.z, ch.y));
    InPlane r;
    if (fabsf(dxk) >= fabsf(dyk)) {
        r.axis = 0;
        const float m = __fmul_rn(__fdiv_rn(dyk, dxk), G.dx_dy);
        r.aq = __fmaf_rn(-vw.x, m, vw.y);
        r.bq = m;
        r.kappa = __fdiv_rn(G.dx_sdd, dxk);
        r.tau0 = __fmul_rn(-vw.x, r.kappa);
        r.Lxy = __fdiv_rn(G.dx, fabsf(dxk));
    } else {
        r.axis = 1;
        const float m = __fmul_rn(__fdiv_rn(dxk, dyk), G.dy_dx);
        r.aq = __fmaf_rn(-vw.y, m, vw.x);
        r.bq = m;
        r.kappa = __fdiv_rn(G.dy_sdd, dyk);
        r.tau0 = __fmul_rn(-vw.y, r.kappa);
        r.Lxy = __fdiv_rn(G.dy, fabsf(dyk));
    }
    return r;
}

// In-plane parameters of (view, channel) read back from the table that
// build_inplane_table filled with ray_inplane(): the forward and backward
// projectors both read it, so their sample positions are identical by construction.
__device__ __forceinline__ InPlane inplane_at(float4 a, float lsigned) {
    InPlane r;
    r.axis = lsigned < 0.f ? 1 : 0;
    r.aq = a.x;
    r.bq = a.y;
    r.tau0 = a.z;
    r.kappa = a.w;
    r.Lxy = fabsf(lsigned);
    return r;
}

// Row height omega_r = w_r / dz of detector row r, in slices: omega0 + r domega,
// one explicitly rounded FMA wherever either projector direction needs it.
__device__ __forceinline__ float row_omega(const Geo& G, int r) { return __fmaf_rn((float)r, G.domega, G.omega0); }

// Ray parameter at plane p (fraction of u from the source): t(p) = tau0 + p kappa.
__device__ __forceinline__ float ray_t(const InPlane& ip, float p) { return __fmaf_rn(p, ip.kappa, ip.tau0); }

// z-intercept (index units) of the ray of row r at ray parameter t:
// fz = sigma_z + omega_r t.  Both projector directions evaluate exactly this
// expression (t from ray_t), so they select the same taps.
__device__ __forceinline__ float row_fz(float sigma_z, float omega, float t) { return __fmaf_rn(omega, t, sigma_z); }

// ---------------------------------------------------------------------------
// kernel launchers (deam_kernels.cu)
// ---------------------------------------------------------------------------
enum BwdMode { BWD_ADJOINT = 0, BWD_UPDATE = 1, BWD_GRADIENT = 2 };
// FWD_DEAM_F32: FWD_DEAM with plain FP32 spectral sums and FP32 objective
// accumulation (the uncompensated variant, for comparison)
enum FwdMode { FWD_LINE = 0, FWD_LINE_G = 1, FWD_DEAM = 2, FWD_MASK = 3, FWD_MAX = 4, FWD_COUNT = 5, FWD_DEAM_F32 = 6 };

struct FwdArgs {
    const float4* volX;   // [nx][nz+2][ny+1] q-paired layout for x-dominant rays
    const float4* volY;   // [ny][nz+2][nx+1] q-paired layout for y-dominant rays
    float2* l_out;        // FWD_LINE(_G): [V][R][K] line integrals (nullable in LINE_G)
    float* g_out;         // FWD_LINE_G: [2][V][R][K] expected counts
    const float* dt;      // FWD_DEAM: d~ [2][V][R][K]
    const uint8_t* mask;  // FWD_DEAM: [V][R][K] metal traces, bit j = spectrum j (nullable: none)
    const float* bowtie;  // [K] (nullable: 1)
    float4* payload;      // FWD_DEAM: [V][R][K] (B~1, B~2, D1, D2)
    double* partial;      // FWD_DEAM: per-block objective; FWD_MAX: per-block max; FWD_COUNT: samples
    uint8_t* mask_out;    // FWD_MASK
    float threshold;      // FWD_MASK
    int fold_rowfac;      // FWD_DEAM: 1 stores the payload times the row length factor (the
                          // backprojector's input form); 0: the payload as defined (deam_ray_terms)
};

struct BwdArgs {
    const float2* rays2;    // BWD_ADJOINT input [V][R][K][2]
    const float4* payload;  // BWD_UPDATE / BWD_GRADIENT input [V][R][K][4]
    float2* img;            // adjoint or gradient output / update in-out c [nz][ny][nx]
    const int2* slab_views; // [n_slabs][tiles y][tiles x] view range [lo, hi] per z-slab and column tile
    double invZ;            // 1 / Z of the c-step
    int clamp_nonneg;
    unsigned long long* skipped;  // update: count of unchanged (voxel, component) pairs
    // regularised c-step (Eqs. 6-7), lambda > 0: the backprojection stores its
    // per-voxel sums in `sums` and reg_update_kernel solves; neighbours' c^k are
    // read from the projector layout volX, which holds c^k while the update runs
    float4* sums;                 // [nvox] (b~_1, b~_2, delta_1, delta_2); nullptr: plain c-step
    float lambda, delta, Z;
    float pdx, pdy, pdz;          // voxel edges (mm) for the 1/distance weights
    const float4* volX;
};

// Batched launch over many scans (deam_batch_*): per-scan descriptors in
// device memory and prefix sums of each scan's work items.
struct BatchDesc {
    int n;                      // scans
    const Geo* geos;            // [n]
    const Spec* specs;          // [n]
    const FwdArgs* fargs;       // [n]
    const BwdArgs* bargs;       // [n] (slab views for the chosen slab depth)
    const long long* ftile_off; // [n+1] prefix sums of forward ray tiles
    const long long* btile_off; // [n+1] prefix sums of backprojection tiles
    double* partial;            // [ftile_off[n]] objective per forward tile
};
// Scan of batch work item t: the last i with off[i] <= t (prefix sums of the
// scans' work items).
__device__ __forceinline__ int find_scan(const long long* off, int n, long long t) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&off[mid]) <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Forward ray-tile and backprojection-tile shapes an autotuner may choose from.
constexpr int kFwdShapes[3][2] = {{8, 1}, {4, 2}, {2, 4}};             // (rows, views) x 32 channels
constexpr int kNumBwdShapes = 6;
constexpr int kBwdShapes[kNumBwdShapes][3] = {{2, 16, 8}, {2, 32, 4}, {8, 16, 8},
                                              {8, 32, 4}, {16, 16, 8}, {16, 32, 4}};  // (slab, tx, ty)
// Slab class of the gather backprojection for a scan: 2 for one or two
// slices, 8 when a detector row covers at most 2/3 of a slice (several rows
// per slot), else 16.  The batched persistent launches use the class as their
// slab depth; a single-scan context runs class 16 as kDeepSlab slices.
inline int pick_slab(int nz, int n_rows, double dz, double row_pitch, double sid, double sdd) {
    if (nz <= 2) return 2;
    return (n_rows == 1 || dz >= 1.5 * row_pitch * sid / sdd) ? 8 : 16;
}
// Slab depth a single-scan context runs for the deep class (16): 13 slices.
// The accumulators of a 128-thread block then take 26 KB of shared memory, so
// with at most 64 registers a thread 8 blocks (32 warps) fit on an SM instead
// of 6: the gather is latency-bound at 6 (measured at 512^2 x 64: 16 slices at
// 6 blocks/SM 203.8 ms, 12 at 7 blocks 193.0 ms, 11 at 8 blocks 189.7 ms).
// The batched persistent launches keep their own shapes (kBwdShapes).
constexpr int kDeepSlab = 13;
inline int context_slab(int slab_class) { return slab_class == 16 ? kDeepSlab : slab_class; }
long long forward_tiles(int shape, const Geo& G);
long long backward_tiles(int shape, const Geo& G);
int forward_batch_blocks_per_sm(int shape);
int backward_batch_blocks_per_sm(int shape);
cudaError_t launch_forward_batch(int shape, const BatchDesc& B, int grid, cudaStream_t s);
cudaError_t launch_backward_batch(int shape, const BatchDesc& B, int grid, cudaStream_t s);
// out[i * stride + *counter] = sum of partial[off[i] .. off[i+1]) (fixed order)
cudaError_t launch_sum_ranges(const double* partial, const long long* off, int n, double* out, const int* counter,
                              int stride, cudaStream_t s);
cudaError_t launch_counter_inc(int* counter, cudaStream_t s);

cudaError_t launch_inplane_table(const Geo& G, float4* ip4, float* ipL, cudaStream_t s);
cudaError_t launch_layout(const float2* c, const float* m, int ones, float4* volX, float4* volY,
                          int nx, int ny, int nz, cudaStream_t s);
int forward_blocks_per_sm();
cudaError_t launch_forward(int mode, const Geo& G, const Spec& S, const FwdArgs& A, int n_blocks,
                           cudaStream_t s);
cudaError_t launch_backward(int mode, int slab, const Geo& G, const BwdArgs& A, cudaStream_t s);
cudaError_t launch_sum_partials(const double* partial, int n, double* out, int do_max, cudaStream_t s);
cudaError_t launch_clamp_copy(const float* d, float* dt, long long n, cudaStream_t s);
cudaError_t launch_mask_bits(uint8_t* m, long long n, int per_spectrum, cudaStream_t s);
cudaError_t launch_reg_update(const Geo& G, const BwdArgs& A, cudaStream_t s);
cudaError_t launch_penalty(const float2* c, int nx, int ny, int nz, float dx, float dy, float dz, float lambda,
                           float delta, double* partial, int n_blocks, cudaStream_t s);
// Measured shared-memory (L1 data path) load throughput of this device, bytes/s.
cudaError_t l1_probe(double* bytes_per_s, cudaStream_t s);
cudaError_t launch_combine(const float2* c, long long nvox, const float2* ab, int n, float* out, cudaStream_t s);

// Record an error message for deam_last_error() and return code (deam_api.cu).
int set_error(int code, const char* msg);
// Validate a scan description on the host: "" if deam_init would accept it,
// else the reason (deam_api.cu).
std::string validate_scan(const deam_geometry* g, const deam_spectra* s, const deam_basis* b);

}  // namespace deam
