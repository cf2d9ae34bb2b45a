// The context behind the opaque deam_ctx handle, shared by the single-scan
// entry points (deam_api.cu) and the batched ones (deam_batch.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "deam.h"
#include "deam_internal.h"

struct deam_ctx {
    deam_geometry geo{};
    deam::Geo G{};
    deam::Spec S{};
    int device = 0;
    double Z = 0.0, threshold = 0.0, mumax = 0.0;
    int clamp = 0;
    double lambda = 0.0, delta = 1.0;  // penalty of Eqs. (6)-(7)
    int fwd_mode = deam::FWD_DEAM;     // FWD_DEAM_F32 for the plain-FP32 variant
    double i0tot[2] = {0.0, 0.0};      // sum_E I0_j(E) (MAR initialisation's log sinograms)
    std::vector<double> energy;        // [n_E] bin centres (keV), empty if not given
    std::vector<double> mu, i0;        // [2][n_E] the caller's attenuation and spectrum tables
    bool has_data = false, mask_set = false, failed = false;
    int batch_refs = 0;                // live batches holding this context (deam_destroy refuses)
    long long nrays = 0, nvox = 0, skipped_last = 0;
    int n_fwd_blocks = 0, n_slabs = 0, slab = 16;
    // device buffers
    float4* view4 = nullptr;
    float* view_z = nullptr;
    float4* ip4 = nullptr;
    float* ipL = nullptr;
    float2* chan = nullptr;
    float2* row = nullptr;
    float* bowtie = nullptr;
    float* dt = nullptr;
    uint8_t* mask = nullptr;
    float4* payload = nullptr;
    float4* volX = nullptr;
    float4* volY = nullptr;
    double* partial = nullptr;
    double* scal = nullptr;  // [0]: last reduction result
    double* hist = nullptr;
    int hist_cap = 0;
    int2* slab_views = nullptr;
    unsigned long long* skipped = nullptr;
    float2* c_stage = nullptr;
    float2* coef = nullptr;  // deam_basis_images coefficients
    float4* sums = nullptr;  // regularised c-step: backprojected sums per voxel (lambda > 0)
    unsigned int* fault = nullptr;  // [2] bounds-checked builds: (site, index) of the first failing access
    // per-kernel timing of deam_iterate (deam_profile)
    bool prof = false;
    double prof_ms[4] = {0, 0, 0, 0};
    long long prof_n[4] = {0, 0, 0, 0};
};

namespace deam {
// View range [lo, hi] whose rays can put a sample into z-slab s of depth slab
// at the columns [ix0, ix1] x [iy0, iy1].
int2 slab_view_range(const deam_geometry& g, int s, int slab, int ix0, int ix1, int iy0, int iy1);
// The ranges of every (slab, tx x ty column tile), slab-major then tile rows:
// the backprojection's work-item order.
std::vector<int2> tile_view_ranges(const deam_geometry& g, int slab, int tx, int ty);
// Projector volume layouts of c (or of the metal image m, or of ones).
int build_layouts(deam_ctx* ctx, const float2* c, const float* m, int ones, cudaStream_t s);
// Forward-kernel arguments bound to the context's buffers.
FwdArgs fwd_args(deam_ctx* ctx);
// Penalty fields of the backprojection arguments (lambda = 0: unregularised).
void set_penalty_args(const deam_ctx* ctx, BwdArgs& B);
// End of an entry point that launched kernels on s: DEAM_OK, or in a
// bounds-checked build DEAM_ERR_ARG when a kernel recorded an out-of-range
// access in the context's fault words (read back and cleared; synchronises s).
int finish_call(deam_ctx* ctx, cudaStream_t s);
}  // namespace deam
