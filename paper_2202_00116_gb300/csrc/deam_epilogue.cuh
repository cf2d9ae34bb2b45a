// Device helpers of the per-ray spectral epilogue (Eq. 8 energy sums and the
// Eq. 5 I-divergence term) and block reductions, shared by the kernels that
// compute them.
#pragma once

#include <math.h>

#include "deam_internal.h"

namespace deam {

// ex2.approx: the SFU's 2^x (documented max relative error 2^-22); the tables
// carry mu * log2(e) so that exp(-mu.l) = 2^(-mu'.l).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Kahan/Neumaier-style compensated accumulation of a block partial.
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float x) {
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// (1 + u) ln(1 + u) - u, the I-divergence term d ln(d/g) - d + g divided by g
// with u = (d - g) / g.  For |u| < 1/4 the Taylor series
// sum_{n>=2} (-1)^n u^n / (n (n-1)) through u^12 (the first dropped term is
// below 3e-9 of the sum) avoids the cancellation of the closed form.  Beyond,
// the closed form with one rounding for (1 + u) ln(1 + u) - u (an FMA): the
// cancellation there amplifies log1pf's error by at most (1+u) ln(1+u) / phi,
// about 10 at |u| = 1/4 and falling with |u|, so each term is within ~2e-6
// (relative) of its exact value; the terms are summed in FP64.
__device__ __forceinline__ float idiv_phi(float u) {
    if (u <= -1.f) return 1.f;  // d = 0: the term is g
    if (fabsf(u) < 0.25f) {
        float s = 1.f / 132.f;
        s = fmaf(s, u, -1.f / 110.f);
        s = fmaf(s, u, 1.f / 90.f);
        s = fmaf(s, u, -1.f / 72.f);
        s = fmaf(s, u, 1.f / 56.f);
        s = fmaf(s, u, -1.f / 42.f);
        s = fmaf(s, u, 1.f / 30.f);
        s = fmaf(s, u, -1.f / 20.f);
        s = fmaf(s, u, 1.f / 12.f);
        s = fmaf(s, u, -1.f / 6.f);
        s = fmaf(s, u, 0.5f);
        return s * u * u;
    }
    return fmaf(1.f + u, log1pf(u), -u);
}

// Sum (or max) over a block of NT threads in a fixed order: warp shuffles,
// then thread 0 combines the warp results in warp order.
template <int NT, typename T>
__device__ __forceinline__ T block_reduce(T v, bool is_max) {
    __shared__ T red[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T w = __shfl_down_sync(0xffffffffu, v, o);
        v = is_max ? (w > v ? w : v) : v + w;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        v = red[0];
        for (int i = 1; i < NT / 32; ++i) v = is_max ? (red[i] > v ? red[i] : v) : v + red[i];
    }
    return v;
}

// Spectral sums of one ray for both spectra: g_j = sum_E I0_j q~, S_ij = sum_E
// mu_i I0_j q~ with q~ = 2^(-mu'.l) (bowtie applied by the caller).  Bins are
// summed in blocks of 8 in FP32, block partials are added with compensation.
// COMP = false: plain FP32 sums, bin after bin (the uncompensated variant).
template <bool NEED_S, bool COMP = true>
__device__ __forceinline__ void spectral_sums(const Spec& S, float l1, float l2, float& gl, float& gh,
                                              float& s1l, float& s2l, float& s1h, float& s2h) {
    float cgl = 0.f, cgh = 0.f, c1l = 0.f, c2l = 0.f, c1h = 0.f, c2h = 0.f;
    gl = gh = s1l = s2l = s1h = s2h = 0.f;
    if constexpr (!COMP) {
        for (int e = S.e_lo; e < S.e_hi; ++e) {
            const float ex = ex2_approx(-fmaf(S.mu1l2[e], l1, S.mu2l2[e] * l2));
            const float ql = S.i0l[e] * ex, qh = S.i0h[e] * ex;
            gl += ql;
            gh += qh;
            if (NEED_S) {
                s1l = fmaf(S.mu1[e], ql, s1l);
                s2l = fmaf(S.mu2[e], ql, s2l);
                s1h = fmaf(S.mu1[e], qh, s1h);
                s2h = fmaf(S.mu2[e], qh, s2h);
            }
        }
    } else {
        for (int e0 = S.e_lo; e0 < S.e_hi; e0 += 8) {
            float pgl = 0.f, pgh = 0.f, p1l = 0.f, p2l = 0.f, p1h = 0.f, p2h = 0.f;
            const int n = min(8, S.e_hi - e0);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (i < n) {
                    const int e = e0 + i;
                    const float ex = ex2_approx(-fmaf(S.mu1l2[e], l1, S.mu2l2[e] * l2));
                    const float ql = S.i0l[e] * ex, qh = S.i0h[e] * ex;
                    pgl += ql;
                    pgh += qh;
                    if (NEED_S) {
                        p1l = fmaf(S.mu1[e], ql, p1l);
                        p2l = fmaf(S.mu2[e], ql, p2l);
                        p1h = fmaf(S.mu1[e], qh, p1h);
                        p2h = fmaf(S.mu2[e], qh, p2h);
                    }
                }
            }
            kahan_add(gl, cgl, pgl);
            kahan_add(gh, cgh, pgh);
            if (NEED_S) {
                kahan_add(s1l, c1l, p1l);
                kahan_add(s2l, c2l, p2l);
                kahan_add(s1h, c1h, p1h);
                kahan_add(s2h, c2h, p2h);
            }
        }
    }
}

}  // namespace deam
