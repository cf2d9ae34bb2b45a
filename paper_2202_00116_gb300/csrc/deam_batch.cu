// Batched MAR-DEAM: many independent scans (each a deam_ctx with its data and
// metal mask set) iterated together.  One iteration is a fixed set of launches
// whatever the number of scans: the per-scan projector layouts, one persistent
// forward launch over the ray tiles of every scan, one launch reducing every
// scan's objective, one persistent backprojection launch per slab class (2, 8
// or 16 slices, from each scan's geometry) over the column tiles of its scans,
// and an iteration counter.  The sequence is captured once in a CUDA graph and
// replayed per iteration.  The ray-tile shape of the forward launch and the
// column-tile shape of each backprojection class are picked by timing every
// candidate on the batch itself (on scratch copies of the images).  A second
// plan records each scan's own single-scan kernels on a graph branch of its
// own (small scans then overlap large ones); the tuner times one captured
// iteration of both plans and keeps the faster.
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

constexpr int kNF = 3;  // forward ray-tile shapes (deam::kFwdShapes)
constexpr int kNB = deam::kNumBwdShapes;  // backprojection shapes (deam::kBwdShapes)
constexpr int kSlabs[3] = {2, 8, 16};     // slab classes

}  // namespace

struct deam_batch {
    int n = 0, device = 0, autotune = 1;
    std::vector<deam_ctx*> ctx;
    bool holds_refs = false;  // the contexts' batch_refs count this batch
    deam::Geo* geos = nullptr;
    deam::Spec* specs = nullptr;
    deam::FwdArgs* fargs = nullptr;
    deam::BwdArgs* bargs[kNB] = {};
    int2* slabviews[kNB] = {};
    long long* foff[kNF] = {};
    long long* boff[kNB] = {};
    std::vector<deam::BwdArgs> hbargs[kNB];
    double* partial = nullptr;
    double* hist = nullptr;
    int hist_cap = 0;
    int* counter = nullptr;
    int fshape = 1;
    int bshape[3] = {-1, -1, -1};   // chosen shape per slab class (-1: no scan in the class)
    long long class_tiles[3] = {0, 0, 0};
    bool tuned = false;
    float tune_fwd_ms[kNF] = {0, 0, 0}, tune_bwd_ms[kNB] = {0, 0, 0, 0, 0, 0};
    int fgrid[kNF] = {}, bgrid[kNB] = {};
    int plan = 0;                    // 0: persistent launches over all scans, 1: per-scan launches on graph branches
    int min_plan = 0;                // 1 when a scan asks for the plain-FP32 forward (plan 0 has only the compensated one)
    float tune_plan_ms[2] = {0, 0};
    long long* soff = nullptr;       // [n][2] = {0, forward blocks of scan i}: per-scan objective ranges
    std::vector<cudaStream_t> br;    // graph branches of the per-scan plan
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaStream_t cs = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<float*> graph_c;
    int graph_cap = 0;
    std::vector<float2*> scratch;
};

#define BK(x)                                                                                   \
    do {                                                                                        \
        cudaError_t e_ = (x);                                                                   \
        if (e_ != cudaSuccess)                                                                  \
            return fail(e_ == cudaErrorMemoryAllocation ? DEAM_ERR_OOM : DEAM_ERR_CUDA,         \
                        std::string(#x) + ": " + cudaGetErrorString(e_));                       \
    } while (0)

static void free_batch(deam_batch* b) {
    if (b->holds_refs)
        for (deam_ctx* x : b->ctx) --x->batch_refs;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cs) cudaStreamDestroy(b->cs);
    for (cudaStream_t q : b->br)
        if (q) cudaStreamDestroy(q);
    for (cudaEvent_t q : b->join)
        if (q) cudaEventDestroy(q);
    if (b->fork) cudaEventDestroy(b->fork);
    void* p[] = {b->geos, b->specs, b->fargs, b->partial, b->hist, b->counter, b->soff};
    for (void* q : p)
        if (q) cudaFree(q);
    for (int s = 0; s < kNB; ++s) {
        if (b->bargs[s]) cudaFree(b->bargs[s]);
        if (b->slabviews[s]) cudaFree(b->slabviews[s]);
        if (b->boff[s]) cudaFree(b->boff[s]);
    }
    for (int s = 0; s < kNF; ++s)
        if (b->foff[s]) cudaFree(b->foff[s]);
    for (float2* q : b->scratch)
        if (q) cudaFree(q);
    delete b;
}

static deam::BatchDesc desc(const deam_batch* b, int fs, int bs) {
    deam::BatchDesc D{};
    D.n = b->n;
    D.geos = b->geos;
    D.specs = b->specs;
    D.fargs = b->fargs;
    D.bargs = b->bargs[bs];
    D.ftile_off = b->foff[fs];
    D.btile_off = b->boff[bs];
    D.partial = b->partial;
    return D;
}

// Point every scan's backprojection arguments at the images to update.
static int set_images(deam_batch* b, const std::vector<float2*>& img, cudaStream_t s) {
    for (int sh = 0; sh < kNB; ++sh) {
        for (int i = 0; i < b->n; ++i) b->hbargs[sh][i].img = img[i];
        BK(cudaMemcpyAsync(b->bargs[sh], b->hbargs[sh].data(), sizeof(deam::BwdArgs) * b->n, cudaMemcpyHostToDevice,
                           s));
    }
    BK(cudaStreamSynchronize(s));
    return DEAM_OK;
}

static int tune_plan(deam_batch* b);

// Time every candidate shape on scratch copies of the images and keep the fastest.
static int tune(deam_batch* b, float* const* c) {
    cudaStream_t s = b->cs;
    if (b->scratch.empty()) {
        b->scratch.assign(b->n, nullptr);
        for (int i = 0; i < b->n; ++i) BK(cudaMalloc((void**)&b->scratch[i], sizeof(float2) * b->ctx[i]->nvox));
    }
    for (int i = 0; i < b->n; ++i)
        BK(cudaMemcpyAsync(b->scratch[i], c[i], sizeof(float2) * b->ctx[i]->nvox, cudaMemcpyDeviceToDevice, s));
    int rc = set_images(b, b->scratch, s);
    if (rc != DEAM_OK) return rc;
    for (int i = 0; i < b->n; ++i) {
        rc = deam::build_layouts(b->ctx[i], b->scratch[i], nullptr, 0, s);
        if (rc != DEAM_OK) return rc;
    }
    cudaEvent_t e0, e1;
    BK(cudaEventCreate(&e0));
    BK(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int fs = 0; fs < kNF; ++fs) {
        float ms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {  // the first run also warms caches
            BK(cudaEventRecord(e0, s));
            BK(deam::launch_forward_batch(fs, desc(b, fs, 0), b->fgrid[fs], s));
            BK(cudaEventRecord(e1, s));
            BK(cudaEventSynchronize(e1));
            float t = 0.f;
            BK(cudaEventElapsedTime(&t, e0, e1));
            ms = std::min(ms, t);
        }
        b->tune_fwd_ms[fs] = ms;
        if (ms < best) {
            best = ms;
            b->fshape = fs;
        }
    }
    // the payload of the last forward run is valid for every backprojection candidate
    BK(deam::launch_forward_batch(b->fshape, desc(b, b->fshape, 0), b->fgrid[b->fshape], s));
    for (int cl = 0; cl < 3; ++cl) {
        if (b->bshape[cl] < 0) continue;
        best = 1e30f;
        for (int bs = 0; bs < kNB; ++bs) {
            if (deam::kBwdShapes[bs][0] != kSlabs[cl]) continue;
            float ms = 1e30f;
            for (int rep = 0; rep < 2; ++rep) {
                BK(cudaEventRecord(e0, s));
                BK(deam::launch_backward_batch(bs, desc(b, b->fshape, bs), b->bgrid[bs], s));
                BK(cudaEventRecord(e1, s));
                BK(cudaEventSynchronize(e1));
                float t = 0.f;
                BK(cudaEventElapsedTime(&t, e0, e1));
                ms = std::min(ms, t);
            }
            b->tune_bwd_ms[bs] = ms;
            if (ms < best) {
                best = ms;
                b->bshape[cl] = bs;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    rc = tune_plan(b);
    if (rc != DEAM_OK) return rc;
    b->tuned = true;
    return DEAM_OK;
}

// Record one iteration of the whole batch on the capturing stream b->cs.
// plan 0: the persistent batched kernels; plan 1: every scan's own kernels
// (the single-scan launches of deam_iterate) on a graph branch of its own.
static int record_iteration(deam_batch* b, float* const* c, int plan) {
    cudaStream_t s = b->cs;
    int rc = DEAM_OK;
    cudaError_t e = cudaSuccess;
    if (plan == 0) {
        for (int i = 0; i < b->n && rc == DEAM_OK; ++i)
            rc = deam::build_layouts(b->ctx[i], (const float2*)c[i], nullptr, 0, s);
        if (rc != DEAM_OK) return rc;
        e = deam::launch_forward_batch(b->fshape, desc(b, b->fshape, 0), b->fgrid[b->fshape], s);
        if (e == cudaSuccess)
            e = deam::launch_sum_ranges(b->partial, b->foff[b->fshape], b->n, b->hist, b->counter, b->hist_cap, s);
        for (int i = 0; i < b->n && e == cudaSuccess; ++i)
            e = cudaMemsetAsync(b->ctx[i]->skipped, 0, sizeof(unsigned long long), s);
        for (int cl = 0; cl < 3 && e == cudaSuccess; ++cl)  // one persistent launch per slab class
            if (b->bshape[cl] >= 0)
                e = deam::launch_backward_batch(b->bshape[cl], desc(b, b->fshape, b->bshape[cl]),
                                                b->bgrid[b->bshape[cl]], s);
        for (int i = 0; i < b->n && e == cudaSuccess; ++i)  // regularised scans: the per-voxel solve
            if (b->ctx[i]->lambda > 0.0) {
                deam::BwdArgs B = b->hbargs[0][i];
                B.img = (float2*)c[i];
                e = deam::launch_reg_update(b->ctx[i]->G, B, s);
            }
    } else {
        e = cudaEventRecord(b->fork, s);
        for (int i = 0; i < b->n && e == cudaSuccess && rc == DEAM_OK; ++i) {
            deam_ctx* x = b->ctx[i];
            cudaStream_t q = b->br[i];
            e = cudaStreamWaitEvent(q, b->fork, 0);
            if (e == cudaSuccess) rc = deam::build_layouts(x, (const float2*)c[i], nullptr, 0, q);
            if (rc != DEAM_OK) break;
            deam::FwdArgs A = deam::fwd_args(x);
            A.dt = x->dt;
            A.mask = x->mask_set ? x->mask : nullptr;
            A.payload = x->payload;
            A.fold_rowfac = 1;  // read by launch_backward
            e = deam::launch_forward(x->fwd_mode, x->G, x->S, A, x->n_fwd_blocks, q);
            if (e == cudaSuccess)
                e = deam::launch_sum_ranges(x->partial, b->soff + 2 * i, 1, b->hist + (size_t)i * b->hist_cap,
                                            b->counter, b->hist_cap, q);
            if (e == cudaSuccess) e = cudaMemsetAsync(x->skipped, 0, sizeof(unsigned long long), q);
            deam::BwdArgs B{};
            B.payload = x->payload;
            B.img = (float2*)c[i];
            B.slab_views = x->slab_views;
            B.invZ = 1.0 / x->Z;
            B.clamp_nonneg = x->clamp;
            B.skipped = x->skipped;
            deam::set_penalty_args(x, B);
            if (e == cudaSuccess) e = deam::launch_backward(deam::BWD_UPDATE, x->slab, x->G, B, q);
            if (e == cudaSuccess && B.sums) e = deam::launch_reg_update(x->G, B, q);
            if (e == cudaSuccess) e = cudaEventRecord(b->join[i], q);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join[i], 0);
        }
        if (rc != DEAM_OK) return rc;
    }
    if (e == cudaSuccess) e = deam::launch_counter_inc(b->counter, s);
    BK(e);
    return DEAM_OK;
}

// Capture one iteration of the whole batch into a CUDA graph.
static int capture(deam_batch* b, float* const* c, int plan) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaStream_t s = b->cs;
    BK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const int rc = record_iteration(b, c, plan);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (rc != DEAM_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    BK(e);
    b->graph_c.assign(c, c + b->n);
    b->graph_cap = b->hist_cap;
    b->plan = plan;
    return DEAM_OK;
}

static int ensure_hist(deam_batch* b, int n_iter) {
    if (b->hist_cap >= n_iter) return DEAM_OK;
    if (b->hist) BK(cudaFree(b->hist));
    b->hist = nullptr;
    b->hist_cap = 0;
    BK(cudaMalloc((void**)&b->hist, sizeof(double) * (size_t)b->n * n_iter));
    b->hist_cap = n_iter;
    return DEAM_OK;
}

// Time one captured iteration of each plan on the scratch images; keep the faster.
static int tune_plan(deam_batch* b) {
    int rc = ensure_hist(b, 4);
    if (rc != DEAM_OK) return rc;
    std::vector<float*> sc(b->n);
    for (int i = 0; i < b->n; ++i) sc[i] = (float*)b->scratch[i];
    cudaEvent_t e0, e1;
    BK(cudaEventCreate(&e0));
    BK(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_plan = b->min_plan;
    for (int plan = b->min_plan; plan < 2; ++plan) {
        rc = capture(b, sc.data(), plan);
        if (rc != DEAM_OK) return rc;
        BK(cudaMemsetAsync(b->counter, 0, sizeof(int), b->cs));
        float ms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            BK(cudaEventRecord(e0, b->cs));
            BK(cudaGraphLaunch(b->exec, b->cs));
            BK(cudaEventRecord(e1, b->cs));
            BK(cudaEventSynchronize(e1));
            float t = 0.f;
            BK(cudaEventElapsedTime(&t, e0, e1));
            ms = std::min(ms, t);
        }
        b->tune_plan_ms[plan] = ms;
        if (ms < best) {
            best = ms;
            best_plan = plan;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    b->plan = best_plan;
    return DEAM_OK;
}

extern "C" {

int deam_batch_create(deam_ctx* const* ctxs, int n, int autotune, deam_batch** out) {
    if (!out) return fail(DEAM_ERR_ARG, "out must not be NULL");
    *out = nullptr;
    if (!ctxs || n < 1 || n > 4096) return fail(DEAM_ERR_ARG, "need 1..4096 contexts");
    if (autotune < 0 || autotune > 2) return fail(DEAM_ERR_ARG, "autotune must be 0, 1 or 2");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(DEAM_ERR_CUDA, "no CUDA device");
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return fail(DEAM_ERR_ARG, "null context in batch");
        if (ctxs[i]->failed) return fail(DEAM_ERR_STATE, "a context failed earlier");
        if (ctxs[i]->device != dev) return fail(DEAM_ERR_ARG, "all contexts must live on the current device");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return fail(DEAM_ERR_ARG, "a context appears twice in the batch");
    }
    deam_batch* b = new deam_batch();
    b->n = n;
    b->device = dev;
    b->autotune = autotune == 1 ? 1 : 0;
    b->ctx.assign(ctxs, ctxs + n);
    for (int i = 0; i < n; ++i)
        if (ctxs[i]->fwd_mode != deam::FWD_DEAM) b->min_plan = 1;
    if (autotune == 2) b->min_plan = 1;  // the per-scan plan, untuned
    b->plan = b->min_plan;
    auto bail = [&](int rc) {
        std::string m = deam_last_error();
        free_batch(b);
        return fail(rc, m);
    };
    std::vector<deam::Geo> G(n);
    std::vector<deam::Spec> S(n);
    std::vector<deam::FwdArgs> F(n);
    for (int i = 0; i < n; ++i) {
        G[i] = ctxs[i]->G;
        S[i] = ctxs[i]->S;
        F[i] = deam::fwd_args(ctxs[i]);
        F[i].dt = ctxs[i]->dt;
        F[i].mask = nullptr;  // set at iterate time (a mask may be set after creation)
        F[i].payload = ctxs[i]->payload;
        F[i].fold_rowfac = 1;  // read by the batched backprojection
    }
    std::vector<long long> off(n + 1);
    long long maxf = 0;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    A(cudaMalloc((void**)&b->geos, sizeof(deam::Geo) * n));
    A(cudaMalloc((void**)&b->specs, sizeof(deam::Spec) * n));
    A(cudaMalloc((void**)&b->fargs, sizeof(deam::FwdArgs) * n));
    A(cudaMalloc((void**)&b->counter, sizeof(int)));
    if (e != cudaSuccess) return bail(fail(DEAM_ERR_OOM, "batch descriptor allocation failed"));
    A(cudaMemcpy(b->geos, G.data(), sizeof(deam::Geo) * n, cudaMemcpyHostToDevice));
    A(cudaMemcpy(b->specs, S.data(), sizeof(deam::Spec) * n, cudaMemcpyHostToDevice));
    A(cudaMemcpy(b->fargs, F.data(), sizeof(deam::FwdArgs) * n, cudaMemcpyHostToDevice));
    for (int fs = 0; fs < kNF; ++fs) {
        off[0] = 0;
        for (int i = 0; i < n; ++i) off[i + 1] = off[i] + deam::forward_tiles(fs, G[i]);
        maxf = std::max(maxf, off[n]);
        A(cudaMalloc((void**)&b->foff[fs], sizeof(long long) * (n + 1)));
        if (e == cudaSuccess)
            A(cudaMemcpy(b->foff[fs], off.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice));
        b->fgrid[fs] = sms * deam::forward_batch_blocks_per_sm(fs);
    }
    A(cudaMalloc((void**)&b->partial, sizeof(double) * std::max<long long>(maxf, 1)));
    std::vector<int> cls(n);
    for (int i = 0; i < n; ++i) {
        const deam_geometry& g = ctxs[i]->geo;
        const int sl = deam::pick_slab(g.nz, g.n_rows, g.dz, g.row_pitch, g.sid, g.sdd);
        cls[i] = sl == 2 ? 0 : (sl == 8 ? 1 : 2);
    }
    for (int bs = 0; bs < kNB; ++bs) {
        const int slab = deam::kBwdShapes[bs][0];
        const int cl = slab == 2 ? 0 : (slab == 8 ? 1 : 2);
        std::vector<int2> sv;
        std::vector<size_t> start(n);
        off[0] = 0;
        for (int i = 0; i < n; ++i) {
            // a scan's backprojection tiles appear only in its own slab class
            off[i + 1] = off[i] + (cls[i] == cl ? deam::backward_tiles(bs, G[i]) : 0);
            start[i] = sv.size();
            const std::vector<int2> r = deam::tile_view_ranges(ctxs[i]->geo, slab, deam::kBwdShapes[bs][1],
                                                               deam::kBwdShapes[bs][2]);
            sv.insert(sv.end(), r.begin(), r.end());
        }
        A(cudaMalloc((void**)&b->boff[bs], sizeof(long long) * (n + 1)));
        A(cudaMalloc((void**)&b->slabviews[bs], sizeof(int2) * sv.size()));
        A(cudaMalloc((void**)&b->bargs[bs], sizeof(deam::BwdArgs) * n));
        if (e != cudaSuccess) break;
        A(cudaMemcpy(b->boff[bs], off.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice));
        A(cudaMemcpy(b->slabviews[bs], sv.data(), sizeof(int2) * sv.size(), cudaMemcpyHostToDevice));
        b->hbargs[bs].resize(n);
        for (int i = 0; i < n; ++i) {
            deam::BwdArgs& a = b->hbargs[bs][i];
            a = deam::BwdArgs{};
            a.payload = ctxs[i]->payload;
            a.slab_views = b->slabviews[bs] + start[i];
            a.invZ = 1.0 / ctxs[i]->Z;
            a.clamp_nonneg = ctxs[i]->clamp;
            a.skipped = ctxs[i]->skipped;
            deam::set_penalty_args(ctxs[i], a);
        }
        b->bgrid[bs] = sms * deam::backward_batch_blocks_per_sm(bs);
        if (off[n] > 0 && (b->bshape[cl] < 0 || deam::kBwdShapes[bs][1] == 16)) b->bshape[cl] = bs;  // default 16x8
        b->class_tiles[cl] = off[n];
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    b->br.assign(n, nullptr);
    b->join.assign(n, nullptr);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&b->br[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) {
        std::vector<long long> so(2 * n);
        for (int i = 0; i < n; ++i) {
            so[2 * i] = 0;
            so[2 * i + 1] = ctxs[i]->n_fwd_blocks;
        }
        e = cudaMalloc((void**)&b->soff, sizeof(long long) * 2 * n);
        if (e == cudaSuccess) e = cudaMemcpy(b->soff, so.data(), sizeof(long long) * 2 * n, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(e == cudaErrorMemoryAllocation ? DEAM_ERR_OOM : DEAM_ERR_CUDA,
                         std::string("batch set-up failed: ") + cudaGetErrorString(e)));
    }
    // default shapes when not tuned: the single-scan kernels' shapes
    b->fshape = 1;
    for (deam_ctx* x : b->ctx) ++x->batch_refs;
    b->holds_refs = true;
    *out = b;
    return DEAM_OK;
}

int deam_batch_iterate(deam_batch* b, float* const* c, int n_iter, double* hist, void* stream) {
    if (!b) return fail(DEAM_ERR_ARG, "null batch");
    if (!c) return fail(DEAM_ERR_ARG, "c must not be NULL");
    if (n_iter < 0) return fail(DEAM_ERR_ARG, "n_iter must be >= 0");
    for (int i = 0; i < b->n; ++i) {
        if (!c[i]) return fail(DEAM_ERR_ARG, "null image in batch");
        if (b->ctx[i]->failed) return fail(DEAM_ERR_STATE, "a context failed earlier");
        if (!b->ctx[i]->has_data) return fail(DEAM_ERR_STATE, "deam_set_data has not been called for every scan");
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, c[i]) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            return fail(DEAM_ERR_ARG, "batch images must be device memory");
        }
    }
    if (n_iter == 0) return DEAM_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    struct Restore {
        int p, d;
        ~Restore() {
            if (p >= 0 && p != d) cudaSetDevice(p);
        }
    } restore{prev, b->device};
    cudaStream_t us = (cudaStream_t)stream;
    BK(cudaStreamSynchronize(us));  // the images are written on the caller's stream
    // masks may have been set after the batch was created
    {
        std::vector<deam::FwdArgs> F(b->n);
        for (int i = 0; i < b->n; ++i) {
            F[i] = deam::fwd_args(b->ctx[i]);
            F[i].dt = b->ctx[i]->dt;
            F[i].mask = b->ctx[i]->mask_set ? b->ctx[i]->mask : nullptr;
            F[i].payload = b->ctx[i]->payload;
            F[i].fold_rowfac = 1;
        }
        BK(cudaMemcpyAsync(b->fargs, F.data(), sizeof(deam::FwdArgs) * b->n, cudaMemcpyHostToDevice, b->cs));
    }
    if (b->autotune && !b->tuned) {
        int rc = tune(b, c);
        if (rc != DEAM_OK) return rc;
    }
    std::vector<float2*> img(b->n);
    for (int i = 0; i < b->n; ++i) img[i] = (float2*)c[i];
    int rc = set_images(b, img, b->cs);
    if (rc != DEAM_OK) return rc;
    rc = ensure_hist(b, n_iter);
    if (rc != DEAM_OK) return rc;
    bool recapture = !b->exec || b->graph_cap != b->hist_cap || (int)b->graph_c.size() != b->n;
    for (int i = 0; i < b->n && !recapture; ++i) recapture = b->graph_c[i] != c[i];
    if (recapture) {
        rc = capture(b, c, b->plan);
        if (rc != DEAM_OK) return rc;
    }
    BK(cudaStreamSynchronize(b->cs));
    BK(cudaMemsetAsync(b->counter, 0, sizeof(int), us));
    for (int it = 0; it < n_iter; ++it) BK(cudaGraphLaunch(b->exec, us));
    std::vector<double> h((size_t)b->n * b->hist_cap);
    BK(cudaMemcpyAsync(h.data(), b->hist, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, us));
    BK(cudaStreamSynchronize(us));
    bool finite = true;
    for (int i = 0; i < b->n; ++i)
        for (int it = 0; it < n_iter; ++it) {
            const double v = h[(size_t)i * b->hist_cap + it];
            if (hist) hist[(size_t)i * n_iter + it] = v;
            finite = finite && isfinite(v);
        }
    for (int i = 0; i < b->n; ++i) {  // bounds-checked builds: any recorded out-of-range access
        const int rc = deam::finish_call(b->ctx[i], us);
        if (rc != DEAM_OK) return rc;
    }
    if (!finite) return fail(DEAM_ERR_NUMERIC, "objective became non-finite");
    return DEAM_OK;
}

int deam_batch_info(deam_batch* b, int* plan, float* plan_ms, int* fwd_shape, int* bwd_shapes, float* fwd_ms,
                    float* bwd_ms) {
    if (!b) return fail(DEAM_ERR_ARG, "null batch");
    if (plan) *plan = b->plan;
    if (plan_ms) memcpy(plan_ms, b->tune_plan_ms, sizeof(b->tune_plan_ms));
    if (fwd_shape) {
        fwd_shape[0] = deam::kFwdShapes[b->fshape][0];
        fwd_shape[1] = deam::kFwdShapes[b->fshape][1];
    }
    if (bwd_shapes)
        for (int cl = 0; cl < 3; ++cl)
            for (int j = 0; j < 3; ++j)
                bwd_shapes[3 * cl + j] = b->bshape[cl] >= 0 ? deam::kBwdShapes[b->bshape[cl]][j] : 0;
    if (fwd_ms) memcpy(fwd_ms, b->tune_fwd_ms, sizeof(b->tune_fwd_ms));
    if (bwd_ms) memcpy(bwd_ms, b->tune_bwd_ms, sizeof(b->tune_bwd_ms));
    return DEAM_OK;
}

int deam_batch_destroy(deam_batch* b) {
    if (!b) return DEAM_OK;
    cudaSetDevice(b->device);
    if (b->cs) cudaStreamSynchronize(b->cs);
    cudaDeviceSynchronize();
    free_batch(b);
    return DEAM_OK;
}

}  // extern "C"
