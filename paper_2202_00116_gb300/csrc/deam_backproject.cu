// Voxel-driven gather backprojection of the MAR-DEAM c-step (arXiv 2202.00116,
// Sec. 2.3): b~_i(x) = sum_y h(x,y) B~_i(y) and delta_i(x) = sum_y h(x,y) D_i(y)
// per voxel, fused with the log-ratio update c_i <- c_i - (1/Z) ln(b^_i / b~_i);
// the gradient b^ - b~; and the plain transpose A^T y of two-component ray data.
// h is Joseph's; the gather recomputes the forward kernel's samples exactly, so
// the weights are the forward's transposed and no atomics are needed.
#include <math.h>

#include "deam_internal.h"

namespace deam {

// Voxel-driven gather backprojection.  A block owns a kTileX x kTileY tile of
// (ix, iy) columns and a z-slab of SLAB voxels; each thread owns one column and
// keeps its SLAB accumulators in shared memory (layout [slot][thread], so a
// warp's accesses to one slot are conflict-free).  For every view that can reach
// the slab, the thread takes the channels whose rays can touch its column (fan
// angle of the column centre +- the footprint), evaluates each such ray's sample
// at its plane exactly as the forward kernel does (same in-plane table, same
// explicitly rounded t(p), omega_r and fz), and for every row whose sample falls
// in the slab adds h(x, y) * payload(y) to the two voxels the sample
// interpolates.  The kernel lives on the L1/shared-memory data path (the
// accumulator read-modify-writes and the payload gathers) and on the latency
// of its gathers, so the row loop reads nothing but the payload: omega_r is
// computed, and the payload already carries h's row length factor.  Views are taken in pairs: the samples of one row from
// two consecutive views lie within a few hundredths of a slice of each other,
// so they almost always fall in the same slot pair, and one read-modify-write
// of each slot adds both (half the accumulator traffic).  With 8-slice slabs
// (several rows per slice) consecutive rows share a slot pair instead, which
// is kept in registers.
constexpr int kBwdThreads = kTileX * kTileY;

__device__ __forceinline__ float channel_coord(const Geo& G, float4 vw, float x, float y, float* dist) {
    const float px = (x - vw.x) * G.dx, py = (y - vw.y) * G.dy;
    const float dot = -(px * vw.z + py * vw.w);
    const float crs = px * vw.w - py * vw.z;
    if (dist) *dist = sqrtf(dot * dot + crs * crs);
    return fmaf(atan2f(crs, dot), G.inv_dgamma, G.chan_c0);
}

template <bool FOUR, int SLAB, int NT>
__device__ __forceinline__ void pend_flush(float4* acc, int s, int tid, float4 x) {
    if (s >= 0 && s < SLAB) {
        float4& a = acc[s * NT + tid];
        a.x += x.x;
        a.y += x.y;
        if (FOUR) {
            a.z += x.z;
            a.w += x.w;
        }
    }
}


// One ray's visit of a column: what the row loop needs.
struct ColRay {
    long long pb;  // ray-data index of row 0: (v R) K + k
    float sz;      // sigma_z of the view
    float tp;      // ray parameter at the column's plane
    float Lq;      // Joseph length x in-plane bilinear weight (0: the ray misses the column)
    int r0, r1;    // rows whose sample can land in the slab (r0 > r1: none)
};

// Channel window [k0, k1] of view v for the column at (fix, fiy) (k0 > k1:
// none), and the view's sigma_z.
__device__ __forceinline__ void view_window(const Geo& G, int v, float fix, float fiy, int& k0, int& k1, float& sz) {
    const float4 vw = __ldg(&G.view4[v]);
    sz = __ldg(&G.view_z[v]);
    float dist;
    const float uc = channel_coord(G, vw, fix, fiy, &dist);
    // a ray can tap the column only if it passes within one voxel edge of its
    // centre: |gamma - gamma_c| < asin(edge / dist) < reach / (dist - reach);
    // 0.05 channel of margin covers the FP32 channel coordinate
    const float hw = __fdividef(G.vox_reach_mm, fmaxf(dist - G.vox_reach_mm, 1.f)) * G.inv_dgamma + 0.05f;
    k0 = max(0, (int)ceilf(fmaxf(uc - hw, -1.f)));
    k1 = min(G.K - 1, (int)floorf(fminf(uc + hw, (float)G.K)));
    if (!DEAM_IN_BOUNDS(G, k0 > k1 || (k0 >= 0 && (long long)v * G.K + k1 < (long long)G.V * G.K), SITE_BWD_TABLE,
                        (long long)v * G.K + k1))
        k1 = k0 - 1;
}

__device__ __forceinline__ ColRay no_ray() {
    ColRay c;
    c.pb = 0;
    c.sz = 0.f;
    c.tp = 0.f;
    c.Lq = 0.f;
    c.r0 = 0;
    c.r1 = -1;
    return c;
}

// Ray (v, k) at column (ix, iy), from its in-plane table entry (a4, aL): the
// sample at the column's plane exactly as the forward kernel evaluates it;
// Lq = 0 when the ray does not touch the column.
__device__ __forceinline__ ColRay col_ray(const Geo& G, int v, int k, float4 a4, float aL, int ix, int iy, float sz,
                                          float zlo, float zhi) {
    ColRay c;
    c.pb = (long long)v * G.R * G.K + k;
    c.sz = sz;
    c.Lq = 0.f;
    c.tp = 0.f;
    c.r0 = 0;
    c.r1 = -1;
    const InPlane ip = inplane_at(a4, aL);
    const int p = ip.axis ? iy : ix;
    const int q = ip.axis ? ix : iy;
    const float pf = (float)p;
    const float fq = __fmaf_rn(pf, ip.bq, ip.aq);
    const float jq = floorf(fq);
    const float aq = fq - jq;
    float wq = 0.f;
    if (jq == (float)q) wq = 1.f - aq;
    else if (jq == (float)(q - 1)) wq = aq;
    c.tp = ray_t(ip, pf);
    if (wq == 0.f) return c;
    int r0 = 0, r1 = G.R - 1;
    if (G.R > 1) {
        const float slope = c.tp * G.domega;
        if (fabsf(slope) > 1e-20f) {
            const float inv = __fdividef(1.f, slope);
            const float base = fmaf(c.tp, G.omega0, sz);
            const float ra = (zlo - base) * inv, rb = (zhi - base) * inv;
            const float lo = fminf(fmaxf(fminf(ra, rb), -4.f), (float)G.R + 4.f);
            const float hi = fminf(fmaxf(fmaxf(ra, rb), -4.f), (float)G.R + 4.f);
            r0 = max(0, (int)floorf(lo - 0.02f));
            r1 = min(G.R - 1, (int)ceilf(hi + 0.02f));
        }
    }
    if (!DEAM_IN_BOUNDS(G, c.pb + (long long)(G.R - 1) * G.K < (long long)G.V * G.R * G.K, SITE_BWD_RAY,
                        c.pb + (long long)(G.R - 1) * G.K))
        return c;
    c.Lq = ip.Lxy * wq;
    c.r0 = r0;
    c.r1 = r1;
    return c;
}

template <int MODE>
__device__ __forceinline__ float4 ray_payload(const BwdArgs& A, long long i) {
    if (MODE == BWD_ADJOINT) {
        const float2 t = __ldg(&A.rays2[i]);
        return make_float4(t.x, t.y, 0.f, 0.f);
    }
    float4 P = __ldg(&A.payload[i]);
    if (MODE == BWD_GRADIENT) P = make_float4(P.z, P.w, 0.f, 0.f);
    return P;
}

template <bool FOUR, int SLAB, int NT>
__device__ __forceinline__ void slot_add(float4* acc, int s, int tid, float w, const float4& P) {
    if (s >= 0 && s < SLAB) {
        float4& a = acc[s * NT + tid];
        a.x = fmaf(w, P.x, a.x);
        a.y = fmaf(w, P.y, a.y);
        if (FOUR) {
            a.z = fmaf(w, P.z, a.z);
            a.w = fmaf(w, P.w, a.w);
        }
    }
}

template <bool FOUR, int SLAB, int NT>
__device__ __forceinline__ void slot_add2(float4* acc, int s, int tid, float wa, const float4& Pa, float wb,
                                          const float4& Pb) {
    if (s >= 0 && s < SLAB) {
        float4& a = acc[s * NT + tid];
        a.x = fmaf(wb, Pb.x, fmaf(wa, Pa.x, a.x));
        a.y = fmaf(wb, Pb.y, fmaf(wa, Pa.y, a.y));
        if (FOUR) {
            a.z = fmaf(wb, Pb.z, fmaf(wa, Pa.z, a.z));
            a.w = fmaf(wb, Pb.w, fmaf(wa, Pa.w, a.w));
        }
    }
}

// Rows of two rays of consecutive views at one column.  Their samples of a row
// lie within a few hundredths of a slice of each other, so they nearly always
// fall in the same slot pair: one read-modify-write of each slot serves both.
template <int MODE, int SLAB, int NT>
__device__ __forceinline__ void rows_pair(const Geo& G, const BwdArgs& A, float4* acc, int tid, int z0,
                                          const ColRay& a, const ColRay& b) {
    constexpr bool FOUR = MODE == BWD_UPDATE;
    const int r0 = min(a.r0, b.r0), r1 = max(a.r1, b.r1);
    // not unrolled: within the 64 registers of the 8-blocks-per-SM bound an
    // unrolled body spills (measured 3 % slower at 512^2 x 64)
#pragma unroll 1
    for (int r = r0; r <= r1; ++r) {
        const float4 Pa = ray_payload<MODE>(A, a.pb + (long long)r * G.K);
        const float4 Pb = ray_payload<MODE>(A, b.pb + (long long)r * G.K);
        const float om = row_omega(G, r);
        const float fza = row_fz(a.sz, om, a.tp), fzb = row_fz(b.sz, om, b.tp);
        const float jza = floorf(fza), jzb = floorf(fzb);
        const float aza = fza - jza, azb = fzb - jzb;
        const int sa = (int)jza - z0, sb = (int)jzb - z0;
        const float rf = MODE == BWD_ADJOINT ? __ldg(&G.row[r]).y : 1.f;
        const float wa = a.Lq * rf, wb = b.Lq * rf;
        const float w1a = wa * aza, w0a = wa - w1a;
        const float w1b = wb * azb, w0b = wb - w1b;
        if (sa == sb) {
            slot_add2<FOUR, SLAB, NT>(acc, sa, tid, w0a, Pa, w0b, Pb);
            slot_add2<FOUR, SLAB, NT>(acc, sa + 1, tid, w1a, Pa, w1b, Pb);
        } else {
            slot_add<FOUR, SLAB, NT>(acc, sa, tid, w0a, Pa);
            slot_add<FOUR, SLAB, NT>(acc, sa + 1, tid, w1a, Pa);
            slot_add<FOUR, SLAB, NT>(acc, sb, tid, w0b, Pb);
            slot_add<FOUR, SLAB, NT>(acc, sb + 1, tid, w1b, Pb);
        }
    }
}

// One (column tile, z-slab) of the gather backprojection: the work of one block.
template <int MODE, int SLAB, int TX, int TY>
__device__ __forceinline__ void bwd_tile(const Geo& G, const BwdArgs& A, float4* acc, int bx, int by, int slab) {
    // MODE: BWD_ADJOINT (A^T of two-component ray data), BWD_UPDATE (payload ->
    // b~, delta -> c-step), BWD_GRADIENT (payload -> delta = b^ - b~ = dF/dc)
    constexpr bool FOUR = MODE == BWD_UPDATE;
    constexpr int NT = TX * TY;
    const int tid = threadIdx.x;
    const int ix = bx * TX + (tid % TX);
    const int iy = by * TY + (tid / TX);
    if (ix >= G.nx || iy >= G.ny) return;  // no block-wide synchronisation below
    const int z0 = slab * SLAB;
#pragma unroll
    for (int s = 0; s < SLAB; ++s) acc[s * NT + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    // views that can reach this column tile's slab (host-computed per tile)
    const int2 vrange =
        __ldg(&A.slab_views[((long long)slab * ((G.ny + TY - 1) / TY) + by) * ((G.nx + TX - 1) / TX) + bx]);
    const float fix = (float)ix, fiy = (float)iy;
    const float zlo = (float)(z0 - 1), zhi = (float)(z0 + SLAB);
    if constexpr (SLAB != 8) {
        // views in pairs (v, v + 1): the j-th channel of one with the j-th of the other
        for (int v = vrange.x; v <= vrange.y; v += 2) {
            int ka0, ka1, kb0 = 0, kb1 = -1;
            float sza, szb = 0.f;
            view_window(G, v, fix, fiy, ka0, ka1, sza);
            if (v + 1 <= vrange.y) view_window(G, v + 1, fix, fiy, kb0, kb1, szb);
            const int nj = max(ka1 - ka0, kb1 - kb0) + 1;
            for (int j = 0; j < nj; ++j) {
                ColRay a = no_ray(), b = no_ray();
                if (ka0 + j <= ka1) {
                    const long long i = (long long)v * G.K + ka0 + j;
                    a = col_ray(G, v, ka0 + j, __ldg(&G.ip4[i]), __ldg(&G.ipL[i]), ix, iy, sza, zlo, zhi);
                }
                if (kb0 + j <= kb1) {
                    const long long i = (long long)(v + 1) * G.K + kb0 + j;
                    b = col_ray(G, v + 1, kb0 + j, __ldg(&G.ip4[i]), __ldg(&G.ipL[i]), ix, iy, szb, zlo, zhi);
                }
                if (a.Lq == 0.f && b.Lq == 0.f) continue;
                // a missing partner: the other ray with zero weight (same slots, same loads)
                if (a.Lq == 0.f) {
                    a = b;
                    a.Lq = 0.f;
                }
                if (b.Lq == 0.f) {
                    b = a;
                    b.Lq = 0.f;
                }
                rows_pair<MODE, SLAB, NT>(G, A, acc, tid, z0, a, b);
            }
        }
    } else {
        for (int v = vrange.x; v <= vrange.y; ++v) {
            int k0, k1;
            float sz;
            view_window(G, v, fix, fiy, k0, k1, sz);
            const long long vbase = (long long)v * G.K;
            float4 na = make_float4(0.f, 0.f, 0.f, 0.f);
            float nl = 1.f;
            if (k0 <= k1) {
                na = __ldg(&G.ip4[vbase + k0]);
                nl = __ldg(&G.ipL[vbase + k0]);
            }
            for (int k = k0; k <= k1; ++k) {
                const InPlane ip = inplane_at(na, nl);
                if (k < k1) {  // prefetch the next channel's parameters
                    na = __ldg(&G.ip4[vbase + k + 1]);
                    nl = __ldg(&G.ipL[vbase + k + 1]);
                }
                const int p = ip.axis ? iy : ix;
                const int q = ip.axis ? ix : iy;
                const float pf = (float)p;
                const float fq = __fmaf_rn(pf, ip.bq, ip.aq);
                const float jq = floorf(fq);
                const float aq = fq - jq;
                float wq;
                if (jq == (float)q) wq = 1.f - aq;
                else if (jq == (float)(q - 1)) wq = aq;
                else continue;
                if (wq == 0.f) continue;
                const float tp = ray_t(ip, pf);  // ray parameter at plane p
                int r0 = 0, r1 = G.R - 1;
                if (G.R > 1) {
                    // fz(r) = sigma_z + t (omega0 + r domega): rows whose sample can
                    // land in [z0 - 1, z0 + SLAB).  Solved in FP32 with the fast
                    // reciprocal (within ~1e-6 rows of the rounded samples); a
                    // 0.02-row margin keeps every contributing row, and the exact
                    // per-row slot test below decides.
                    const float slope = tp * G.domega;
                    if (fabsf(slope) > 1e-20f) {
                        const float inv = __fdividef(1.f, slope);
                        const float base = fmaf(tp, G.omega0, sz);
                        const float ra = (zlo - base) * inv, rb = (zhi - base) * inv;
                        const float lo = fminf(fmaxf(fminf(ra, rb), -4.f), (float)G.R + 4.f);
                        const float hi = fminf(fmaxf(fmaxf(ra, rb), -4.f), (float)G.R + 4.f);
                        r0 = max(0, (int)floorf(lo - 0.02f));
                        r1 = min(G.R - 1, (int)ceilf(hi + 0.02f));
                    }
                }
                const float Lq = ip.Lxy * wq;
                // two or more rows fall in one slice, so consecutive rows add to the
                // same slot pair: keep it in registers (plo: slot ls, phi: slot
                // ls + 1) and write shared memory when the slot moves on
                float4 plo = make_float4(0.f, 0.f, 0.f, 0.f), phi = plo;
                int ls = -1000;
                // ray data [V][R][K]: a warp's columns read neighbouring channels of a row
                const long long pb = vbase * G.R + k;
                if (!DEAM_IN_BOUNDS(G, pb + (long long)r1 * G.K < (long long)G.V * G.R * G.K, SITE_BWD_RAY,
                                    pb + (long long)r1 * G.K))
                    continue;
    #pragma unroll 4
                for (int r = r0; r <= r1; ++r) {
                    float4 Pv;
                    if (MODE == BWD_ADJOINT) {
                        const float2 t = __ldg(&A.rays2[pb + (long long)r * G.K]);
                        Pv = make_float4(t.x, t.y, 0.f, 0.f);
                    } else {
                        Pv = __ldg(&A.payload[pb + (long long)r * G.K]);
                        if (MODE == BWD_GRADIENT) Pv = make_float4(Pv.z, Pv.w, 0.f, 0.f);
                    }
                    const float fz = row_fz(sz, row_omega(G, r), tp);
                    const float jz = floorf(fz);
                    const float az = fz - jz;
                    const int sl = (int)jz - z0;
                    // the payload carries h's row length factor already (folded by
                    // the forward kernel); A^T of caller data applies it here
                    const float w = MODE == BWD_ADJOINT ? Lq * __ldg(&G.row[r]).y : Lq;
                    const float w1 = w * az, w0 = w - w1;
                    if (sl != ls) {   // slots rise with r: flush the slot that is complete
                        pend_flush<FOUR, SLAB, NT>(acc, ls, tid, plo);
                        if (sl == ls + 1) {
                            plo = phi;
                        } else {
                            pend_flush<FOUR, SLAB, NT>(acc, ls + 1, tid, phi);
                            plo = make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                        phi = make_float4(0.f, 0.f, 0.f, 0.f);
                        ls = sl;
                    }
                    plo.x = fmaf(w0, Pv.x, plo.x);
                    plo.y = fmaf(w0, Pv.y, plo.y);
                    phi.x = fmaf(w1, Pv.x, phi.x);
                    phi.y = fmaf(w1, Pv.y, phi.y);
                    if (FOUR) {
                        plo.z = fmaf(w0, Pv.z, plo.z);
                        plo.w = fmaf(w0, Pv.w, plo.w);
                        phi.z = fmaf(w1, Pv.z, phi.z);
                        phi.w = fmaf(w1, Pv.w, phi.w);
                    }
                }
                pend_flush<FOUR, SLAB, NT>(acc, ls, tid, plo);
                pend_flush<FOUR, SLAB, NT>(acc, ls + 1, tid, phi);
            }
        }
    }

    unsigned long long skipped = 0;
    for (int s = 0; s < SLAB; ++s) {
        const int iz = z0 + s;
        if (iz >= G.nz) break;
        const float4 a = acc[s * NT + tid];
        const long long vi = ((long long)iz * G.ny + iy) * G.nx + ix;
        if (!DEAM_IN_BOUNDS(G, vi < (long long)G.nx * G.ny * G.nz, SITE_BWD_IMAGE, vi)) break;
        if (!FOUR) {  // A^T y, or the gradient delta_i
            A.img[vi] = make_float2(a.x, a.y);
            continue;
        }
        if (A.sums) {  // regularised c-step: reg_update_kernel finishes the update
            A.sums[vi] = a;
            continue;
        }
        float2 c = A.img[vi];
        // c-step: c_i <- c_i - (1/Z) ln(b^_i / b~_i) = c_i - (1/Z) log1p(delta_i / b~_i);
        // the ratio and its logarithm in FP64 (two per voxel and iteration)
        if (a.x > 0.f && a.z > -a.x) {
            c.x = (float)fma(-log1p((double)a.z / (double)a.x), A.invZ, (double)c.x);
            if (A.clamp_nonneg) c.x = fmaxf(c.x, 0.f);
        } else {
            ++skipped;
        }
        if (a.y > 0.f && a.w > -a.y) {
            c.y = (float)fma(-log1p((double)a.w / (double)a.y), A.invZ, (double)c.y);
            if (A.clamp_nonneg) c.y = fmaxf(c.y, 0.f);
        } else {
            ++skipped;
        }
        A.img[vi] = c;
    }
    if (FOUR && skipped) atomicAdd(A.skipped, skipped);
}



// At most 64 registers a thread: 8 blocks per SM (shared memory allows it up
// to kDeepSlab slices); more resident warps hide the gathers' latency.
template <int MODE, int SLAB>
__global__ void __launch_bounds__(kBwdThreads, 8) bwd_kernel(const Geo G, const BwdArgs A) {
    __shared__ float4 acc[SLAB * kBwdThreads];
    const int ntx = (G.nx + kTileX - 1) / kTileX, nty = (G.ny + kTileY - 1) / kTileY;
    int b = blockIdx.x;
    const int bx = b % ntx;
    b /= ntx;
    const int by = b % nty;
    bwd_tile<MODE, SLAB, kTileX, kTileY>(G, A, acc, bx, by, b / nty);
}

// Batched scans: one persistent launch walks the column tiles x slabs of every
// scan of a slab class; each work item finds its scan by binary search in the
// prefix sums of tile counts.
// (the backprojection keeps the scan's descriptors in registers: staging them
// in shared memory was measured slower for this kernel; bounded to the
// single-scan kernel's 6 blocks/SM, which it now meets without spilling)
template <int SLAB, int TX, int TY>
__global__ void __launch_bounds__(TX* TY, 6) bwd_batch_kernel(const BatchDesc B) {
    __shared__ float4 acc[SLAB * TX * TY];
    const long long total = __ldg(&B.btile_off[B.n]);
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        const int i = find_scan(B.btile_off, B.n, t);
        const Geo G = B.geos[i];
        const BwdArgs A = B.bargs[i];
        long long lt = t - __ldg(&B.btile_off[i]);
        const int ntx = (G.nx + TX - 1) / TX, nty = (G.ny + TY - 1) / TY;
        const int bx = (int)(lt % ntx);
        lt /= ntx;
        const int by = (int)(lt % nty);
        bwd_tile<BWD_UPDATE, SLAB, TX, TY>(G, A, acc, bx, by, (int)(lt / nty));
    }
}


cudaError_t launch_backward(int mode, int slab, const Geo& G, const BwdArgs& A, cudaStream_t s) {
    const int ntx = (G.nx + kTileX - 1) / kTileX, nty = (G.ny + kTileY - 1) / kTileY;
    const int nsl = (G.nz + slab - 1) / slab;
    const int blocks = ntx * nty * nsl;
#define DEAM_BWD(M, SL) bwd_kernel<M, SL><<<blocks, kBwdThreads, 0, s>>>(G, A)
    if (slab == 2) {
        if (mode == BWD_UPDATE) DEAM_BWD(BWD_UPDATE, 2);
        else if (mode == BWD_GRADIENT) DEAM_BWD(BWD_GRADIENT, 2);
        else DEAM_BWD(BWD_ADJOINT, 2);
    } else if (slab == 8) {
        if (mode == BWD_UPDATE) DEAM_BWD(BWD_UPDATE, 8);
        else if (mode == BWD_GRADIENT) DEAM_BWD(BWD_GRADIENT, 8);
        else DEAM_BWD(BWD_ADJOINT, 8);
    } else if (slab == kDeepSlab) {
        if (mode == BWD_UPDATE) DEAM_BWD(BWD_UPDATE, kDeepSlab);
        else if (mode == BWD_GRADIENT) DEAM_BWD(BWD_GRADIENT, kDeepSlab);
        else DEAM_BWD(BWD_ADJOINT, kDeepSlab);
    } else {
        return cudaErrorInvalidValue;
    }
#undef DEAM_BWD
    return cudaGetLastError();
}

long long backward_tiles(int shape, const Geo& G) {
    const int slab = kBwdShapes[shape][0], tx = kBwdShapes[shape][1], ty = kBwdShapes[shape][2];
    return (long long)((G.nx + tx - 1) / tx) * ((G.ny + ty - 1) / ty) * ((G.nz + slab - 1) / slab);
}


#define DEAM_BWD_BATCH_SHAPES(X) \
    X(0, 2, 16, 8) X(1, 2, 32, 4) X(2, 8, 16, 8) X(3, 8, 32, 4) X(4, 16, 16, 8) X(5, 16, 32, 4)

int backward_batch_blocks_per_sm(int shape) {
    int nb = 1;
#define X(I, SL, TX, TY) \
    if (shape == I) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bwd_batch_kernel<SL, TX, TY>, TX * TY, 0);
    DEAM_BWD_BATCH_SHAPES(X)
#undef X
    return nb > 0 ? nb : 1;
}


cudaError_t launch_backward_batch(int shape, const BatchDesc& B, int grid, cudaStream_t s) {
#define X(I, SL, TX, TY) \
    if (shape == I) {    \
        bwd_batch_kernel<SL, TX, TY><<<grid, TX * TY, 0, s>>>(B); \
        return cudaGetLastError(); \
    }
    DEAM_BWD_BATCH_SHAPES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace deam
