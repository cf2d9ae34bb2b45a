// MAR initialisation (Sec. 2.2, Eq. 4): log sinograms, LI / NMAR completion of
// the metal trace, equiangular fan-beam / helical FDK-style filtered
// backprojection, the thresholded prior and the image-domain decomposition.
// These run once per scan, before the DEAM iterations; every step is a
// data-parallel kernel here (the prior's projection reuses the Joseph forward
// kernel).  Declarations and conventions: include/deam.h.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "deam.h"
#include "deam_ctx.h"
#include "deam_internal.h"

namespace {

int fail(int code, const std::string& m) { return deam::set_error(code, m.c_str()); }

const double kPi = 3.14159265358979323846;

#define CK(x)                                                                                  \
    do {                                                                                       \
        cudaError_t e_ = (x);                                                                  \
        if (e_ != cudaSuccess) {                                                               \
            ctx->failed = true;                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? DEAM_ERR_OOM : DEAM_ERR_CUDA,        \
                        std::string(#x) + ": " + cudaGetErrorString(e_));                      \
        }                                                                                      \
    } while (0)

#define CHECK_READY(ctx)                                                                   \
    do {                                                                                   \
        if (!(ctx)) return fail(DEAM_ERR_ARG, "null context");                             \
        if ((ctx)->failed) return fail(DEAM_ERR_STATE, "context failed earlier");          \
        if (!(ctx)->has_data) return fail(DEAM_ERR_STATE, "deam_set_data has not been called"); \
    } while (0)

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// FBP constants (rounded once from double on the host).
struct FbpGeo {
    int nx, ny, nz, V, R, K;
    float x0, y0, z0, dx, dy, dz;  // voxel centres x0 + i dx (mm)
    float inv_da, kc, kmax;        // channel coordinate = gamma / a + kc, valid in [0, kmax]
    float sdd, inv_rp, rc;         // row coordinate = w / row_pitch + rc
    float dbeta;                   // 2 pi / views per rotation
};

// The ramp filter keeps a zero-padded row (3K floats) and the kernel (K floats)
// in shared memory: 16 K bytes within the default 48 KB per block.
constexpr int kMaxFbpChannels = 3072;

int grid_for(long long n, int threads) {
    return (int)std::max<long long>(1, std::min<long long>((n + threads - 1) / threads, 152LL * 32));
}

// ---- kernels -----------------------------------------------------------------

// p_j(y) = ln(I0_j b(k) / max(d~_j(y), floor)), both spectra.
__global__ void log_kernel(const float* __restrict__ dt, const float* __restrict__ bowtie, float i0l, float i0h,
                           float floor_c, long long nrays, int K, float* __restrict__ p) {
    for (long long y = (long long)blockIdx.x * blockDim.x + threadIdx.x; y < nrays;
         y += (long long)gridDim.x * blockDim.x) {
        const float b = bowtie ? bowtie[y % K] : 1.f;
        const float dl = fmaxf(dt[y], floor_c), dh = fmaxf(dt[nrays + y], floor_c);
        p[y] = logf(__fdiv_rn(i0l * b, dl));
        p[nrays + y] = logf(__fdiv_rn(i0h * b, dh));
    }
}

// Linear interpolation across the trace along each (view, row); one block per
// row, the row's (normalised) values and trace flags staged in shared memory.
// In place (out == p) is safe: a thread writes only its own channels and reads
// neighbours from shared memory.
template <bool PRIOR>
__global__ void trace_kernel(const float* p, const float* __restrict__ prior, int pstride,
                             const uint8_t* __restrict__ mask, int bit, float eps, int K, long long nrows, float* out) {
    extern __shared__ float sm[];
    float* nv = sm;
    unsigned char* on = (unsigned char*)(sm + K);
    for (long long row = blockIdx.x; row < nrows; row += gridDim.x) {
        const long long base = row * K;
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            const float pk = p[base + k];
            on[k] = (mask[base + k] >> bit) & 1;
            nv[k] = PRIOR ? __fdiv_rn(pk, fmaxf(prior[(base + k) * pstride], eps)) : pk;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            if (!on[k]) {
                out[base + k] = p[base + k];
                continue;
            }
            int kl = k - 1, kr = k + 1;
            while (kl >= 0 && on[kl]) --kl;
            while (kr < K && on[kr]) ++kr;
            float val;
            if (kl >= 0 && kr < K)
                val = fmaf(nv[kr] - nv[kl], __fdiv_rn((float)(k - kl), (float)(kr - kl)), nv[kl]);
            else if (kl >= 0)
                val = nv[kl];
            else if (kr < K)
                val = nv[kr];
            else
                val = nv[k];
            out[base + k] = PRIOR ? val * fmaxf(prior[(base + k) * pstride], eps) : val;
        }
        __syncthreads();
    }
}

// Equiangular ramp filtering of each (view, row): the pre-weighted row (fan
// weight SID cos(gamma_k), cone weight per row) between zero padding in shared
// memory, q(n) = sum_m ker(|m|) pw(n - m), ker(0) and the odd taps only (the
// even taps vanish), compensated FP32 sums (the taps cancel strongly).  One
// block per row; in place is safe (the row is staged before it is written).
__global__ void ramp_kernel(const float* p, const float* __restrict__ chanw, const float* __restrict__ conew,
                            const float* __restrict__ ker, int K, int R, long long nrows, float* out) {
    extern __shared__ float sm[];
    float* pw = sm;          // [3K]: zeros | weighted row | zeros
    float* kk = sm + 3 * K;  // [K]
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        kk[k] = ker[k];
        pw[k] = 0.f;
        pw[2 * K + k] = 0.f;
    }
    for (long long row = blockIdx.x; row < nrows; row += gridDim.x) {
        const float cw = conew[row % R];
        __syncthreads();  // the previous row's readers are done
        for (int k = threadIdx.x; k < K; k += blockDim.x) pw[K + k] = p[row * K + k] * chanw[k] * cw;
        __syncthreads();
        for (int n = threadIdx.x; n < K; n += blockDim.x) {
            float s = kk[0] * pw[K + n], c = 0.f;
            for (int m = 1; m < K; m += 2) {
                const float y = fmaf(kk[m], pw[K + n - m] + pw[K + n + m], -c);
                const float t = s + y;
                c = (t - s) - y;
                s = t;
            }
            out[row * K + n] = s;
        }
    }
}

// Voxel-driven FBP backprojection of NS filtered sinograms: one thread per
// voxel, one block row per (iy, iz) so that the view window (per slice) is
// uniform in the block; weight 1/L^2, bilinear in (row, channel).
template <int NS>
__global__ void fbp_kernel(const float* __restrict__ q, long long nrays, const float4* __restrict__ vw,
                           const float* __restrict__ vz, const int2* __restrict__ win, const FbpGeo F,
                           float* __restrict__ img) {
    const int ix = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y, iz = blockIdx.z;
    if (ix >= F.nx) return;
    const float X = fmaf((float)ix, F.dx, F.x0), Y = fmaf((float)iy, F.dy, F.y0), Z = fmaf((float)iz, F.dz, F.z0);
    const int2 w = win[iz];
    float acc[NS], cmp[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] = cmp[s] = 0.f;
    for (int v = w.x; v < w.y; ++v) {
        const float4 sv = __ldg(&vw[v]);  // (s_x, s_y, cos beta, sin beta)
        const float ddx = X - sv.x, ddy = Y - sv.y;
        const float L2 = fmaf(ddx, ddx, ddy * ddy);
        // fan angle of the voxel: signed angle from the central ray -(cos, sin)
        const float dot = -fmaf(ddx, sv.z, ddy * sv.w);
        const float crs = fmaf(ddx, sv.w, -ddy * sv.z);
        const float kf = fmaf(atan2f(crs, dot), F.inv_da, F.kc);
        if (!(kf >= 0.f && kf <= F.kmax)) continue;
        const int k0 = min((int)kf, F.K - 2);
        const float ak = kf - (float)k0;
        int r0 = 0;
        float ar = 0.f;
        if (F.R > 1) {
            const float wd = __fdiv_rn((Z - __ldg(&vz[v])) * F.sdd, sqrtf(L2));
            const float rf = fminf(fmaxf(fmaf(wd, F.inv_rp, F.rc), 0.f), (float)(F.R - 1));
            r0 = min((int)rf, F.R - 2);
            ar = rf - (float)r0;
        }
        const float inv = __frcp_rn(L2);
        const long long e = ((long long)v * F.R + r0) * F.K + k0;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const float* qs = q + s * nrays;
            float val = fmaf(ak, __ldg(&qs[e + 1]) - __ldg(&qs[e]), __ldg(&qs[e]));
            if (F.R > 1) {
                const float hi = fmaf(ak, __ldg(&qs[e + F.K + 1]) - __ldg(&qs[e + F.K]), __ldg(&qs[e + F.K]));
                val = fmaf(ar, hi - val, val);
            }
            const float y = fmaf(val, inv, -cmp[s]);
            const float t = acc[s] + y;
            cmp[s] = (t - acc[s]) - y;
            acc[s] = t;
        }
    }
    const long long nvox = (long long)F.nx * F.ny * F.nz;
    const long long vi = ((long long)iz * F.ny + iy) * F.nx + ix;
#pragma unroll
    for (int s = 0; s < NS; ++s) img[s * nvox + vi] = acc[s] * F.dbeta;
}

// One pass of the in-plane [1,2,1]/4 x [1,2,1]/4 smoothing (edges replicated).
__global__ void smooth_kernel(const float* __restrict__ f, int nx, int ny, long long n, float* __restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nx), iy = (int)((i / nx) % ny);
        const long long base = i - ix - (long long)iy * nx;
        float acc = 0.f;
#pragma unroll
        for (int b = -1; b <= 1; ++b) {
            const int y = min(max(iy + b, 0), ny - 1);
            const float wy = b == 0 ? 0.5f : 0.25f;
#pragma unroll
            for (int a = -1; a <= 1; ++a) {
                const int x = min(max(ix + a, 0), nx - 1);
                const float wx = a == 0 ? 0.5f : 0.25f;
                acc = fmaf(wx * wy, f[base + (long long)y * nx + x], acc);
            }
        }
        out[i] = acc;
    }
}

__global__ void prior_kernel(const float* __restrict__ f, long long n, float t_air, float t_bone, float soft,
                             float* __restrict__ prior) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float x = f[i];
        prior[i] = x < t_air ? 0.f : (x < t_bone ? soft : x);
    }
}

// Eq. (4): (c_1, c_2) = M^-1 (mu_L, mu_H), M^-1 rounded once from double.
__global__ void decompose_kernel(const float* __restrict__ mu, long long n, float a, float b, float c, float d,
                                 float2* __restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float l = mu[i], h = mu[n + i];
        out[i] = make_float2(fmaf(a, l, b * h), fmaf(c, l, d * h));
    }
}

// ---- host helpers ------------------------------------------------------------

// prior (nullable): the prior's projection, element y at prior[y * pstride].
int complete(deam_ctx* ctx, const float* p, const float* prior, int pstride, int bit, float eps, float* out,
             cudaStream_t s) {
    const deam_geometry& g = ctx->geo;
    const long long nrows = (long long)g.n_views * g.n_rows;
    const int K = g.n_channels;
    if (!ctx->mask_set) {  // no trace: a copy
        if (out != p) CK(cudaMemcpyAsync(out, p, sizeof(float) * ctx->nrays, cudaMemcpyDeviceToDevice, s));
        return DEAM_OK;
    }
    const size_t sm = sizeof(float) * K + K;
    const int blocks = (int)std::min<long long>(nrows, 152LL * 16);
    if (prior)
        trace_kernel<true><<<blocks, 256, sm, s>>>(p, prior, pstride, ctx->mask, bit, eps, K, nrows, out);
    else
        trace_kernel<false><<<blocks, 256, sm, s>>>(p, nullptr, 1, ctx->mask, bit, eps, K, nrows, out);
    CK(cudaGetLastError());
    return DEAM_OK;
}

// FBP of n sinograms p [n][V][R][K] into img [n][nz][ny][nx]; q is scratch of
// the same size as p (may equal p when p may be overwritten).
int fbp(deam_ctx* ctx, const float* p, int n, float* q, float* img, cudaStream_t s) {
    const deam_geometry& g = ctx->geo;
    const int K = g.n_channels, R = g.n_rows, V = g.n_views, N = g.views_per_rotation;
    // host tables in double, rounded once
    std::vector<float> ker(K), chanw(K), conew(R), vz(V);
    std::vector<float4> vw(V);
    std::vector<int2> win(g.nz);
    const double a = g.channel_pitch;
    for (int m = 0; m < K; ++m) {
        double v;
        if (m == 0) v = 1.0 / (8.0 * a * a);
        else if (m % 2 == 0) v = 0.0;
        else {
            const double sn = sin(m * a);
            v = -1.0 / (2.0 * kPi * kPi * sn * sn);
        }
        ker[m] = (float)(a * v);
    }
    for (int k = 0; k < K; ++k)
        chanw[k] = (float)(g.sid * cos((k - (K - 1) / 2.0 + g.channel_offset) * a));
    for (int r = 0; r < R; ++r) {
        const double w = (r - (R - 1) / 2.0 + g.row_offset) * g.row_pitch;
        conew[r] = (float)(g.sdd / sqrt(g.sdd * g.sdd + w * w));
    }
    for (int v = 0; v < V; ++v) {
        const double beta = g.start_angle + 2.0 * kPi * v / N;
        vw[v] = make_float4((float)(g.sid * cos(beta)), (float)(g.sid * sin(beta)), (float)cos(beta),
                            (float)sin(beta));
        vz[v] = (float)(g.z_start + g.feed * (double)v / N);
    }
    const double Z0 = g.cz - (g.nz - 1) / 2.0 * g.dz;
    for (int iz = 0; iz < g.nz; ++iz) {
        long lo = 0, hi = V < N ? V : N;
        if (g.feed != 0.0 && R > 1) {
            const double vc = (Z0 + iz * g.dz - g.z_start) * (double)N / g.feed;
            lo = (long)ceil(vc - N / 2.0);
            hi = lo + N;
        }
        lo = std::max<long>(lo, 0);
        hi = std::min<long>(hi, V);
        win[iz] = make_int2((int)lo, (int)std::max(lo, hi));
    }
    FbpGeo F;
    F.nx = g.nx; F.ny = g.ny; F.nz = g.nz; F.V = V; F.R = R; F.K = K;
    F.x0 = (float)(g.cx - (g.nx - 1) / 2.0 * g.dx);
    F.y0 = (float)(g.cy - (g.ny - 1) / 2.0 * g.dy);
    F.z0 = (float)Z0;
    F.dx = (float)g.dx; F.dy = (float)g.dy; F.dz = (float)g.dz;
    F.inv_da = (float)(1.0 / a);
    F.kc = (float)((K - 1) / 2.0 - g.channel_offset);
    F.kmax = (float)(K - 1);
    F.sdd = (float)g.sdd;
    F.inv_rp = (float)(1.0 / g.row_pitch);
    F.rc = (float)((R - 1) / 2.0 - g.row_offset);
    F.dbeta = (float)(2.0 * kPi / N);

    // one scratch block for the tables
    const size_t off_ker = 0, off_chw = off_ker + K, off_cone = off_chw + K, off_vz = off_cone + R;
    const size_t nfl = off_vz + V;
    const size_t bytes_fl = ((nfl * sizeof(float) + 15) / 16) * 16;
    const size_t bytes = bytes_fl + sizeof(float4) * V + sizeof(int2) * g.nz;
    char* tab = nullptr;
    CK(cudaMallocAsync((void**)&tab, bytes, s));
    std::vector<char> host(bytes);
    memcpy(host.data() + off_ker * 4, ker.data(), 4 * K);
    memcpy(host.data() + off_chw * 4, chanw.data(), 4 * K);
    memcpy(host.data() + off_cone * 4, conew.data(), 4 * R);
    memcpy(host.data() + off_vz * 4, vz.data(), 4 * V);
    memcpy(host.data() + bytes_fl, vw.data(), sizeof(float4) * V);
    memcpy(host.data() + bytes_fl + sizeof(float4) * V, win.data(), sizeof(int2) * g.nz);
    cudaError_t e = cudaMemcpyAsync(tab, host.data(), bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host staging buffer goes out of scope
    const float* d_ker = (const float*)tab + off_ker;
    const float* d_chw = (const float*)tab + off_chw;
    const float* d_cone = (const float*)tab + off_cone;
    const float* d_vz = (const float*)tab + off_vz;
    const float4* d_vw = (const float4*)(tab + bytes_fl);
    const int2* d_win = (const int2*)(tab + bytes_fl + sizeof(float4) * V);
    const long long nrows = (long long)V * R;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        ramp_kernel<<<(int)std::min<long long>(nrows, 152LL * 8), 256, sizeof(float) * 4 * K, s>>>(
            p + (size_t)i * ctx->nrays, d_chw, d_cone, d_ker, K, R, nrows, q + (size_t)i * ctx->nrays);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const dim3 grid((g.nx + 127) / 128, g.ny, g.nz);
        if (n == 2) fbp_kernel<2><<<grid, 128, 0, s>>>(q, ctx->nrays, d_vw, d_vz, d_win, F, img);
        else fbp_kernel<1><<<grid, 128, 0, s>>>(q, ctx->nrays, d_vw, d_vz, d_win, F, img);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaFreeAsync(tab, s);
    CK(e);
    CK(e2);
    return DEAM_OK;
}

bool is_dev(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

int deam_log_sinogram(deam_ctx* ctx, double count_floor, float* p, void* stream) {
    CHECK_READY(ctx);
    if (!p || !is_dev(p)) return fail(DEAM_ERR_ARG, "p must be a device pointer");
    if (!(isfinite(count_floor) && count_floor > 0.0)) return fail(DEAM_ERR_ARG, "count_floor must be > 0");
    DevGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    log_kernel<<<grid_for(ctx->nrays, 256), 256, 0, s>>>(ctx->dt, ctx->bowtie, (float)ctx->i0tot[0],
                                                         (float)ctx->i0tot[1], (float)count_floor, ctx->nrays,
                                                         ctx->geo.n_channels, p);
    CK(cudaGetLastError());
    return DEAM_OK;
}

int deam_complete_trace(deam_ctx* ctx, const float* p, const float* prior_proj, int spectrum, double eps, float* out,
                        void* stream) {
    CHECK_READY(ctx);
    if (!p || !out || !is_dev(p) || !is_dev(out)) return fail(DEAM_ERR_ARG, "p and out must be device pointers");
    if (prior_proj && !is_dev(prior_proj)) return fail(DEAM_ERR_ARG, "prior_proj must be a device pointer");
    if (spectrum != 0 && spectrum != 1) return fail(DEAM_ERR_ARG, "spectrum must be 0 (L) or 1 (H)");
    if (!(isfinite(eps) && eps > 0.0)) return fail(DEAM_ERR_ARG, "eps must be > 0");
    DevGuard dg(ctx->device);
    return complete(ctx, p, prior_proj, 1, spectrum, (float)eps, out, (cudaStream_t)stream);
}

int deam_fbp(deam_ctx* ctx, const float* p, int n, float* img, void* stream) {
    CHECK_READY(ctx);
    if (n != 1 && n != 2) return fail(DEAM_ERR_ARG, "n must be 1 or 2");
    if (!p || !img || !is_dev(p) || !is_dev(img)) return fail(DEAM_ERR_ARG, "p and img must be device pointers");
    if (ctx->geo.n_channels < 2 || ctx->geo.n_channels > kMaxFbpChannels)
        return fail(DEAM_ERR_ARG, "FBP needs 2 to 3072 channels (the ramp filter stages a row in shared memory)");
    DevGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    float* q = nullptr;
    CK(cudaMallocAsync((void**)&q, sizeof(float) * ctx->nrays * n, s));
    const int rc = fbp(ctx, p, n, q, img, s);
    cudaFreeAsync(q, s);
    return rc;
}

int deam_mar_init(deam_ctx* ctx, const deam_mar_params* P, const float* prior_in, float* c, float* prior_out,
                  float* mu_out, void* stream) {
    CHECK_READY(ctx);
    if (!P || !c || !is_dev(c)) return fail(DEAM_ERR_ARG, "params and a device c are required");
    if ((prior_in && !is_dev(prior_in)) || (prior_out && !is_dev(prior_out)) || (mu_out && !is_dev(mu_out)))
        return fail(DEAM_ERR_ARG, "prior_in, prior_out and mu_out must be device pointers (or NULL)");
    for (double x : {P->calib[0], P->calib[1], P->calib[2], P->calib[3], P->t_air, P->t_bone, P->soft_value})
        if (!isfinite(x)) return fail(DEAM_ERR_ARG, "MAR parameters must be finite");
    const double det = P->calib[0] * P->calib[3] - P->calib[1] * P->calib[2];
    const double scale = std::max(std::fabs(P->calib[0] * P->calib[3]), std::fabs(P->calib[1] * P->calib[2]));
    if (!(std::fabs(det) > 1e-12 * scale)) return fail(DEAM_ERR_ARG, "calibration matrix is singular");
    if (!(isfinite(P->count_floor) && P->count_floor > 0.0)) return fail(DEAM_ERR_ARG, "count_floor must be > 0");
    if (!(isfinite(P->eps) && P->eps > 0.0)) return fail(DEAM_ERR_ARG, "eps must be > 0");
    if (P->prior_spectrum != 0 && P->prior_spectrum != 1) return fail(DEAM_ERR_ARG, "prior_spectrum must be 0 or 1");
    if (P->prior_smooth < 0 || P->prior_smooth > 16) return fail(DEAM_ERR_ARG, "prior_smooth must be 0..16");
    if (ctx->geo.n_channels < 2 || ctx->geo.n_channels > kMaxFbpChannels)
        return fail(DEAM_ERR_ARG, "FBP needs 2 to 3072 channels (the ramp filter stages a row in shared memory)");
    DevGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const long long nr = ctx->nrays, nv = ctx->nvox;
    float *p = nullptr, *t = nullptr, *img = nullptr;
    float2* l = nullptr;
    // p: both sinograms; t: completed sinograms (filtered in place);
    // img: f | prior | mu_L | mu_H | smoothing scratch
    CK(cudaMallocAsync((void**)&p, sizeof(float) * 2 * nr, s));
    cudaError_t e = cudaMallocAsync((void**)&t, sizeof(float) * 2 * nr, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&img, sizeof(float) * 5 * nv, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&l, sizeof(float2) * nr, s);
    auto release = [&]() {
        if (p) cudaFreeAsync(p, s);
        if (t) cudaFreeAsync(t, s);
        if (img) cudaFreeAsync(img, s);
        if (l) cudaFreeAsync(l, s);
    };
    auto run = [&]() -> int {
        CK(e);
        float* f = img;
        float* prior = img + nv;
        float* mu = img + 2 * nv;
        log_kernel<<<grid_for(nr, 256), 256, 0, s>>>(ctx->dt, ctx->bowtie, (float)ctx->i0tot[0],
                                                     (float)ctx->i0tot[1], (float)P->count_floor, nr,
                                                     ctx->geo.n_channels, p);
        CK(cudaGetLastError());
        if (prior_in) {
            CK(cudaMemcpyAsync(prior, prior_in, sizeof(float) * nv, cudaMemcpyDeviceToDevice, s));
        } else {
            // single-energy FBP of the chosen spectrum with the trace linearly
            // interpolated, thresholded into the prior
            const int j = P->prior_spectrum;
            int rc = complete(ctx, p + (size_t)j * nr, nullptr, 1, j, (float)P->eps, t, s);
            if (rc != DEAM_OK) return rc;
            rc = fbp(ctx, t, 1, t, f, s);
            if (rc != DEAM_OK) return rc;
            // filtering: passes ping-pong between f and the scratch image
            float* a = f;
            float* b = img + 4 * nv;  // smoothing scratch
            for (int pass = 0; pass < P->prior_smooth; ++pass) {
                smooth_kernel<<<grid_for(nv, 256), 256, 0, s>>>(a, ctx->geo.nx, ctx->geo.ny, nv, b);
                CK(cudaGetLastError());
                std::swap(a, b);
            }
            prior_kernel<<<grid_for(nv, 256), 256, 0, s>>>(a, nv, (float)P->t_air, (float)P->t_bone,
                                                           (float)P->soft_value, prior);
            CK(cudaGetLastError());
        }
        // the prior's projection: Joseph forward projection of (prior, 0) into
        // l (float2 per ray; NMAR reads its first component)
        int rc = deam::build_layouts(ctx, nullptr, prior, 0, s);
        if (rc != DEAM_OK) return rc;
        deam::FwdArgs A = deam::fwd_args(ctx);
        A.l_out = l;
        CK(deam::launch_forward(deam::FWD_LINE, ctx->G, ctx->S, A, ctx->n_fwd_blocks, s));
        for (int j = 0; j < 2; ++j) {
            rc = complete(ctx, p + (size_t)j * nr, (const float*)l, 2, j, (float)P->eps, t + (size_t)j * nr, s);
            if (rc != DEAM_OK) return rc;
        }
        rc = fbp(ctx, t, 2, t, mu, s);  // both spectra, filtered in place
        if (rc != DEAM_OK) return rc;
        const double ia = P->calib[3] / det, ib = -P->calib[1] / det, ic = -P->calib[2] / det, id = P->calib[0] / det;
        decompose_kernel<<<grid_for(nv, 256), 256, 0, s>>>(mu, nv, (float)ia, (float)ib, (float)ic, (float)id,
                                                           (float2*)c);
        CK(cudaGetLastError());
        if (prior_out) CK(cudaMemcpyAsync(prior_out, prior, sizeof(float) * nv, cudaMemcpyDeviceToDevice, s));
        if (mu_out) CK(cudaMemcpyAsync(mu_out, mu, sizeof(float) * 2 * nv, cudaMemcpyDeviceToDevice, s));
        return DEAM_OK;
    };
    int rc = run();
    release();
    return rc;
}

}  // extern "C"
