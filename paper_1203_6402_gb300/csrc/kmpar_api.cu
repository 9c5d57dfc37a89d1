// kmpar_api.cu -- the C ABI of include/kmpar.h: argument checks, context
// buffers, the call order of Algorithm 2 (Bahmani et al., Sec. 3.3) and Lloyd's
// loop.  Every step of the path runs in the kernels of this library.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>

#include "kmpar_internal.cuh"

struct kmpar_ctx {
    kmp::Ctx c;
};

namespace {

thread_local std::string g_err;

kmpar_status fail(kmp::Ctx *c, kmpar_status s, const std::string &msg) {
    if (c) c->err = msg; else g_err = msg;
    return s;
}

kmpar_status cuda_fail(kmp::Ctx *c, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? KMPAR_ERR_OOM : KMPAR_ERR_CUDA, m);
}

#define KMP_CUDA(ctx, expr, where)                          \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, where); \
    } while (0)

bool precision_supported(int p, int d) {
    if (p == KMPAR_FP32) return true;
    const int fmt = kmp::tc::tc_format(p, d);
    return fmt >= 0 && kmp::tc::tc_supported(d, fmt);
}

// A positive integer from the environment (0 when unset or malformed).
uint64_t env_limit(const char *name) {
    const char *v = getenv(name);
    if (!v || !*v) return 0;
    char *end = nullptr;
    const unsigned long long x = strtoull(v, &end, 10);
    return (end && *end == 0) ? (uint64_t)x : 0;
}

int round_capacity(double ell) {
    double c = ell + 10.0 * sqrt(ell) + 64.0;
    if (c > 2.0e9) c = 2.0e9;
    int cap = (int)ceil(c);
    // KMPAR_ROUND_CAPACITY lowers the per-round capacity (fault injection: a round
    // that draws more returns KMPAR_ERR_CAPACITY)
    const uint64_t lim = env_limit("KMPAR_ROUND_CAPACITY");
    if (lim > 0 && lim < (uint64_t)cap) cap = (int)lim;
    return cap;
}

// Context buffers come from one stream-ordered memory pool per device, owned by
// the library.  Its release threshold is unbounded, so the memory a destroyed
// context freed stays mapped for the next context: creating and destroying a
// context then maps no pages and, unlike cudaFree, does not synchronise the device.
// kmpar_release_cached_memory hands the unused part back to the driver.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

cudaError_t ctx_pool(int dev, cudaMemPool_t *out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

// count elements of T on the context's stream, in whole 256-byte units; the bulk
// and vector copies of the kernels need 16-byte aligned buffers
// KMPAR_CTX_LIMIT_BYTES caps the device memory one context may hold (read at every
// allocation; fault injection: an allocation past it fails as out of memory,
// without asking the driver).
template <typename T>
cudaError_t alloc(kmp::Ctx &c, T **p, size_t count) {
    *p = nullptr;
    cudaMemPool_t pool;
    cudaError_t e = ctx_pool(c.dev, &pool);
    if (e != cudaSuccess) return e;
    const size_t bytes = (sizeof(T) * (count ? count : 1) + 255) & ~(size_t)255;
    const uint64_t lim = env_limit("KMPAR_CTX_LIMIT_BYTES");
    if (lim > 0 && c.alloc_bytes + bytes > lim) return cudaErrorMemoryAllocation;
    void *q = nullptr;
    if ((e = cudaMallocFromPoolAsync(&q, bytes, pool, c.stream)) != cudaSuccess) return e;
    if (reinterpret_cast<uintptr_t>(q) & 15u) {
        cudaFreeAsync(q, c.stream);
        return cudaErrorMisalignedAddress;
    }
    *p = static_cast<T *>(q);
    c.alloc_bytes += bytes;
    return cudaSuccess;
}

void free_ctx(kmp::Ctx &c) {
    void *bufs[] = {c.st, c.D2, c.idx, c.drawn, c.cand, c.C, c.w, c.rD2, c.chosen, c.partials,
                    c.labels[0], c.labels[1], c.perm, c.hist, c.base, c.cost_dev, c.tc_img,
                    c.tc_cmax, c.tc_err, c.cand1, c.fix_rows, c.fix_cnt, c.dmin, c.tc_ximg, c.tc_xnorm,
                    c.piece, c.psum, c.rc_cmass, c.rc_sync, c.rc_err, c.chunk, c.tc_v2,
                    c.tc_anchor, c.tc_anchor_part, c.lloyd_rec, c.ex_keys, c.ex_ws, c.ex_ties,
                    c.tc_ncol, c.tc_tscale, c.tc_xscale, c.tc_ub, c.tc_cimg, c.tc_cscale, c.tc_thr,
                    c.tc_lst, c.tc_lcnt, c.fix_rows2, c.fix_cnt2, c.rCT, c.wl_lab[0], c.wl_lab[1], c.rs_buf,
                    c.ll_ub, c.ll_lb, c.ll_rows, c.ll_cnt, c.ll_cold, c.ll_drift, c.ll_other};
    // stream-ordered: the memory returns to the pool once the context's work is done
    for (void *b : bufs)
        if (b) cudaFreeAsync(b, c.stream);
}

int sort_pow2(int cap) {
    int P = 1;
    while (P < cap) P <<= 1;
    return P;
}

}  // namespace

namespace kmp {
// kernels configured once per process (dynamic shared memory above 48 KB)
cudaError_t configure_kernels(int max_sort_pow2, int k);

std::atomic<long long> g_launches{0};

void set_thread_error(const std::string &m) { g_err = m; }

cudaError_t timing_begin(Ctx &c, cudaEvent_t *a) {
    *a = nullptr;
    if (!c.timing) return cudaSuccess;
    cudaError_t e;
    if (c.event_pool.empty()) {
        cudaEvent_t ev;
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return e;
        c.event_pool.push_back(ev);
    }
    *a = c.event_pool.back();
    c.event_pool.pop_back();
    return cudaEventRecord(*a, c.stream);
}

cudaError_t timing_end(Ctx &c, cudaEvent_t a, int cls) {
    if (!c.timing || !a) return cudaSuccess;
    cudaError_t e;
    if (c.event_pool.empty()) {
        cudaEvent_t ev;
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return e;
        c.event_pool.push_back(ev);
    }
    cudaEvent_t b = c.event_pool.back();
    c.event_pool.pop_back();
    c.pending.push_back({a, b, cls});
    return cudaEventRecord(b, c.stream);
}

cudaError_t timing_drain(Ctx &c) {
    for (auto &p : c.pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, p.a, p.b);
        if (e != cudaSuccess) return e;
        c.kernel_ms[p.cls] += ms;
        c.kernel_launches[p.cls] += 1;
        c.event_pool.push_back(p.a);
        c.event_pool.push_back(p.b);
    }
    c.pending.clear();
    return cudaSuccess;
}
}  // namespace kmp

extern "C" {

const char *kmpar_status_string(kmpar_status s) {
    switch (s) {
        case KMPAR_OK: return "ok";
        case KMPAR_ERR_ARG: return "invalid argument";
        case KMPAR_ERR_CUDA: return "CUDA error";
        case KMPAR_ERR_OOM: return "out of device memory";
        case KMPAR_ERR_CAPACITY: return "round drew more points than its capacity";
        case KMPAR_ERR_TIMEOUT: return "device-side wait timed out";
        case KMPAR_ERR_STATE: return "call out of order";
        case KMPAR_WARN_FEW_CANDIDATES: return "reclustering ran out of positive mass before k draws";
        case KMPAR_ERR_UNSUPPORTED: return "unsupported precision or size";
    }
    return "unknown status";
}

const char *kmpar_last_error(const kmpar_ctx *ctx) { return ctx ? ctx->c.err.c_str() : g_err.c_str(); }

kmpar_status kmpar_init(kmpar_ctx **out, const float *X, int64_t n, int32_t d, int32_t k, double ell,
                        int32_t rounds, uint64_t seed, int32_t precision, void *stream) {
    if (!out) return fail(nullptr, KMPAR_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!X) return fail(nullptr, KMPAR_ERR_ARG, "X is NULL");
    if (n < 1 || n >= (int64_t)INT32_MAX) return fail(nullptr, KMPAR_ERR_ARG, "n out of range [1, 2^31)");
    if (d < 1 || d > 4096) return fail(nullptr, KMPAR_ERR_ARG, "d out of range [1, 4096]");
    if (k < 1) return fail(nullptr, KMPAR_ERR_ARG, "k must be >= 1");
    if (!(ell > 0.0) || !isfinite(ell)) return fail(nullptr, KMPAR_ERR_ARG, "ell must be finite and > 0");
    if (rounds < 0 || rounds > kmp::kMaxRounds) return fail(nullptr, KMPAR_ERR_ARG, "rounds out of range [0, 64]");
    if (!precision_supported(precision, d))
        return fail(nullptr, KMPAR_ERR_UNSUPPORTED, "precision not built into this library for this d");
    const int cap_round = round_capacity(ell);
    if (cap_round > kmp::kMaxRoundCap)
        return fail(nullptr, KMPAR_ERR_UNSUPPORTED, "l + 10 sqrt(l) + 64 exceeds the per-round capacity 32768");
    const int64_t cap_total64 = 1 + (int64_t)rounds * cap_round;
    if (cap_total64 >= INT32_MAX) return fail(nullptr, KMPAR_ERR_ARG, "candidate capacity too large");

    kmpar_ctx *h = new kmpar_ctx();
    kmp::Ctx &c = h->c;
    c.X = X; c.n = n; c.d = d; c.k = k; c.ell = ell; c.rounds = rounds; c.seed = seed;
    c.precision = precision; c.stream = (cudaStream_t)stream;
    c.cap_round = cap_round;
    c.cap_total = (int)cap_total64;
    c.sort_block = kmp::sort_block_size(n, k);
    c.nsb = (int)((n + c.sort_block - 1) / c.sort_block);
    c.num_partials = kmp::assign_num_partials(n, d);

    auto bail = [&](kmpar_status s) {
        std::string m = c.err;
        free_ctx(c);
        delete h;
        g_err = m;
        return s;
    };
    cudaError_t e;
#define KMP_INIT_CUDA(expr, where) \
    if ((e = (expr)) != cudaSuccess) return bail(cuda_fail(&c, e, where))
    KMP_INIT_CUDA(cudaGetDevice(&c.dev), "cudaGetDevice");
    KMP_INIT_CUDA(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.dev), "sm count");
    KMP_INIT_CUDA(kmp::configure_kernels(sort_pow2(cap_round), k), "configure kernels");
    KMP_INIT_CUDA(alloc(c, &c.st, 1), "alloc state");
    KMP_INIT_CUDA(alloc(c, &c.D2, n), "alloc D2");
    KMP_INIT_CUDA(alloc(c, &c.idx, n), "alloc idx");
    KMP_INIT_CUDA(alloc(c, &c.drawn, cap_round), "alloc draws");
    KMP_INIT_CUDA(alloc(c, &c.cand, c.cap_total), "alloc candidates");
    KMP_INIT_CUDA(alloc(c, &c.C, (size_t)c.cap_total * d), "alloc candidate rows");
    KMP_INIT_CUDA(alloc(c, &c.w, c.cap_total), "alloc weights");
    // two buffers (alternating draws) of the padded candidate count
    KMP_INIT_CUDA(alloc(c, &c.rD2, 2 * (size_t)((c.cap_total + 31) / 32 * 32)), "alloc recluster D2");
    KMP_INIT_CUDA(alloc(c, &c.chosen, k), "alloc chosen");
    KMP_INIT_CUDA(alloc(c, &c.rc_cmass, 2 * (size_t)((c.cap_total + 31) / 32) + 2048), "alloc recluster masses");
    unsigned char *rc_sync = nullptr;
    KMP_INIT_CUDA(alloc(c, &rc_sync, kmp::recluster_sync_bytes()), "alloc recluster sync");
    c.rc_sync = rc_sync;
    KMP_INIT_CUDA(alloc(c, &c.rc_err, 1), "alloc recluster error");
    KMP_INIT_CUDA(alloc(c, &c.partials, c.num_partials), "alloc partials");
    if (precision != KMPAR_FP32) {
        namespace tc = kmp::tc;
        const int fmt = tc::tc_format(precision, d);
        c.tc_fmt = fmt;
        c.tc_list = fmt != tc::FMT_BF16X3;
        const int rows = std::max(cap_round, k);
        const size_t n128 = (size_t)((n + 127) / 128) * 128;
        KMP_INIT_CUDA(alloc(c, &c.tc_img, tc::tc_image_bytes(d, fmt, rows)), "alloc center tiles");
        KMP_INIT_CUDA(alloc(c, &c.tc_ncol, (size_t)tc::tc_center_tiles(d, fmt, rows) * tc::tc_block_n(d, fmt)),
                      "alloc center norms");
        KMP_INIT_CUDA(alloc(c, &c.tc_tscale, (size_t)tc::tc_center_tiles(d, fmt, rows)), "alloc tile scales");
        KMP_INIT_CUDA(alloc(c, &c.tc_cmax, 1), "alloc cmax");
        KMP_INIT_CUDA(alloc(c, &c.tc_err, 1), "alloc error word");
        KMP_INIT_CUDA(alloc(c, &c.fix_rows, n), "alloc fix-up rows");
        KMP_INIT_CUDA(alloc(c, &c.cand1, n), "alloc screening winners");
        KMP_INIT_CUDA(alloc(c, &c.tc_v2, n), "alloc screening values");
        KMP_INIT_CUDA(alloc(c, &c.tc_ub, n), "alloc row bounds");
        KMP_INIT_CUDA(alloc(c, &c.tc_ximg, tc::tc_points_image_bytes(d, fmt, n)), "alloc points image");
        KMP_INIT_CUDA(alloc(c, &c.tc_xnorm, n128), "alloc point norms");
        KMP_INIT_CUDA(alloc(c, &c.tc_xscale, n128), "alloc point scales");
        if (c.tc_list) {
            KMP_INIT_CUDA(alloc(c, &c.tc_cimg, tc::tc_points_image_bytes(d, fmt, n)), "alloc list image");
            KMP_INIT_CUDA(alloc(c, &c.tc_cscale, n128), "alloc list scales");
            KMP_INIT_CUDA(alloc(c, &c.tc_thr, n128), "alloc list thresholds");
            KMP_INIT_CUDA(alloc(c, &c.tc_lst, (size_t)n * 4 * tc::kListSlots), "alloc lists");
            KMP_INIT_CUDA(alloc(c, &c.tc_lcnt, (size_t)n * 4), "alloc list counts");
            KMP_INIT_CUDA(alloc(c, &c.fix_rows2, n), "alloc exact-scan rows");
            KMP_INIT_CUDA(alloc(c, &c.fix_cnt2, 1), "alloc exact-scan count");
        }
        KMP_INIT_CUDA(alloc(c, &c.tc_anchor, d), "alloc anchor");
        KMP_INIT_CUDA(alloc(c, &c.tc_anchor_part, tc::tc_anchor_scratch_doubles(d)), "alloc anchor sums");
        KMP_INIT_CUDA(tc::launch_anchor(X, n, d, c.tc_anchor_part, c.tc_anchor, c.stream), "anchor");
        KMP_INIT_CUDA(tc::launch_prep_points(X, n, d, fmt, c.tc_anchor, c.tc_ximg, c.tc_xnorm, c.tc_xscale, c.stream),
                      "points image");
        KMP_INIT_CUDA(alloc(c, &c.fix_cnt, 1), "alloc fix-up count");
        KMP_INIT_CUDA(cudaMemsetAsync(c.tc_err, 0, sizeof(int), c.stream), "memset error word");
    }
    KMP_INIT_CUDA(cudaMemsetAsync(c.st, 0, sizeof(kmp::DevState), c.stream), "memset state");
    KMP_INIT_CUDA(kmp::launch_init_first(c), "init kernels");
#undef KMP_INIT_CUDA
    *out = h;
    return KMPAR_OK;
}

static kmpar_status check_timeout(kmp::Ctx &c) {
    if (!c.tc_err) return KMPAR_OK;
    int err = 0;
    KMP_CUDA(&c, cudaMemcpyAsync(&err, c.tc_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "read error word");
    KMP_CUDA(&c, cudaStreamSynchronize(c.stream), "sync");
    if (err) return fail(&c, KMPAR_ERR_TIMEOUT, "a tensor-core pass timed out waiting (code " + std::to_string(err) + ")");
    return KMPAR_OK;
}

kmpar_status kmpar_round(kmpar_ctx *ctx, int32_t i, int64_t *n_added, double *phi) {
    if (!ctx) return fail(nullptr, KMPAR_ERR_ARG, "ctx is NULL");
    kmp::Ctx &c = ctx->c;
    if (i != c.rounds_done + 1 || i > c.rounds)
        return fail(&c, KMPAR_ERR_STATE, "rounds must be called in order 1..rounds");
    if (c.weighted) return fail(&c, KMPAR_ERR_STATE, "round after weight");
    KMP_CUDA(&c, kmp::launch_round(c, i), "round kernels");
    c.rounds_done = i;
    if (n_added || phi) {
        kmp::DevState st;
        KMP_CUDA(&c, cudaMemcpyAsync(&st, c.st, sizeof(st), cudaMemcpyDeviceToHost, c.stream), "read state");
        KMP_CUDA(&c, cudaStreamSynchronize(c.stream), "sync");
        if (st.overflow) return fail(&c, KMPAR_ERR_CAPACITY, "a round drew more points than its capacity");
        kmpar_status ts = check_timeout(c);
        if (ts != KMPAR_OK) return ts;
        if (n_added) *n_added = st.round_added[i - 1];
        if (phi) *phi = st.phi;
    }
    return KMPAR_OK;
}

kmpar_status kmpar_set_sampling(kmpar_ctx *ctx, int32_t mode) {
    if (!ctx) return fail(nullptr, KMPAR_ERR_ARG, "ctx is NULL");
    kmp::Ctx &c = ctx->c;
    if (c.rounds_done > 0) return fail(&c, KMPAR_ERR_STATE, "sampling is set before round 1");
    if (mode != KMPAR_SAMPLE_BERNOULLI && mode != KMPAR_SAMPLE_EXACT)
        return fail(&c, KMPAR_ERR_ARG, "unknown sampling mode");
    if (mode == KMPAR_SAMPLE_EXACT && !(c.ell >= 1.0))
        return fail(&c, KMPAR_ERR_ARG, "exactly-l rounds need l >= 1");
    if (mode == KMPAR_SAMPLE_EXACT) {
        // each buffer once; after a failed call the next one allocates what is missing
        if (!c.ex_keys) KMP_CUDA(&c, alloc(c, &c.ex_keys, (size_t)c.n), "alloc clocks");
        if (!c.ex_ws) {
            unsigned char *ws = nullptr;
            KMP_CUDA(&c, alloc(c, &ws, kmp::exact_work_bytes()), "alloc select state");
            c.ex_ws = ws;
        }
        if (!c.ex_ties) KMP_CUDA(&c, alloc(c, &c.ex_ties, (size_t)kmp::exact_tie_cap()), "alloc tie list");
    }
    c.sampling = mode == KMPAR_SAMPLE_EXACT ? 1 : 0;
    return KMPAR_OK;
}

kmpar_status kmpar_weight(kmpar_ctx *ctx, int64_t *m_out, const int32_t **cand_idx_dev, const int64_t **w_dev) {
    if (!ctx) return fail(nullptr, KMPAR_ERR_ARG, "ctx is NULL");
    kmp::Ctx &c = ctx->c;
    if (c.rounds_done != c.rounds) return fail(&c, KMPAR_ERR_STATE, "weight before the last round");
    KMP_CUDA(&c, kmp::launch_weights(c), "weights kernel");
    kmp::DevState st;
    KMP_CUDA(&c, cudaMemcpyAsync(&st, c.st, sizeof(st), cudaMemcpyDeviceToHost, c.stream), "read state");
    KMP_CUDA(&c, cudaStreamSynchronize(c.stream), "sync");
    KMP_CUDA(&c, kmp::timing_drain(c), "timing");
    if (st.overflow) return fail(&c, KMPAR_ERR_CAPACITY, "a round drew more points than its capacity");
    kmpar_status ts = check_timeout(c);
    if (ts != KMPAR_OK) return ts;
    c.weighted = true;
    if (m_out) *m_out = st.m;
    if (cand_idx_dev) *cand_idx_dev = c.cand;
    if (w_dev) *w_dev = reinterpret_cast<const int64_t *>(c.w);
    return KMPAR_OK;
}

kmpar_status kmpar_recluster(kmpar_ctx *ctx, float *centers_dev) {
    if (!ctx) return fail(nullptr, KMPAR_ERR_ARG, "ctx is NULL");
    kmp::Ctx &c = ctx->c;
    if (!centers_dev) return fail(&c, KMPAR_ERR_ARG, "centers_dev is NULL");
    if (!c.weighted) return fail(&c, KMPAR_ERR_STATE, "recluster before weight");
    if (!c.rCT) {
        // the grid form and the batched form read the candidates transposed
        const size_t nf = c.rs_batch > 0 ? (size_t)((c.cap_total + 31) / 32) * 32 * (c.d + 2)
                                         : kmp::recluster_grid_floats(c);
        if (nf) KMP_CUDA(&c, alloc(c, &c.rCT, nf), "alloc transposed candidates");
    }
    if (c.rs_batch > 0 && !c.rs_buf) {
        unsigned char *b = nullptr;
        KMP_CUDA(&c, alloc(c, &b, kmp::recluster_batch_bytes()), "alloc batched recluster buffer");
        c.rs_buf = b;
    }
    KMP_CUDA(&c, cudaMemsetAsync(&c.st->warn, 0, sizeof(int32_t), c.stream), "memset warn");
    KMP_CUDA(&c, cudaMemsetAsync(c.rc_err, 0, sizeof(int), c.stream), "memset recluster error");
    if (c.rs_batch > 0)
        KMP_CUDA(&c, kmp::launch_recluster_batch(c, centers_dev), "batched recluster");
    else
        KMP_CUDA(&c, kmp::launch_recluster(c, centers_dev), "recluster kernel");
    int32_t warn = 0, rerr = 0;
    KMP_CUDA(&c, cudaMemcpyAsync(&warn, &c.st->warn, sizeof(warn), cudaMemcpyDeviceToHost, c.stream), "read warn");
    KMP_CUDA(&c, cudaMemcpyAsync(&rerr, c.rc_err, sizeof(rerr), cudaMemcpyDeviceToHost, c.stream), "read error");
    KMP_CUDA(&c, cudaStreamSynchronize(c.stream), "sync");
    if (rerr) return fail(&c, KMPAR_ERR_TIMEOUT, "recluster grid barrier timed out (code " + std::to_string(rerr) + ")");
    return warn ? KMPAR_WARN_FEW_CANDIDATES : KMPAR_OK;
}

kmpar_status kmpar_weighted_lloyd(kmpar_ctx *ctx, float *centers_dev, int32_t max_iter, int32_t *iters) {
    if (!ctx) return fail(nullptr, KMPAR_ERR_ARG, "ctx is NULL");
    kmp::Ctx &c = ctx->c;
    if (!centers_dev) return fail(&c, KMPAR_ERR_ARG, "centers_dev is NULL");
    if (max_iter < 0) return fail(&c, KMPAR_ERR_ARG, "max_iter < 0");
    if (!c.weighted) return fail(&c, KMPAR_ERR_STATE, "weighted Lloyd before weight");
    if (c.d > 4096) return fail(&c, KMPAR_ERR_UNSUPPORTED, "weighted Lloyd supports d <= 4096");
    for (int b = 0; b < 2; ++b)
        if (!c.wl_lab[b]) KMP_CUDA(&c, alloc(c, &c.wl_lab[b], (size_t)c.cap_total), "alloc candidate labels");
    int32_t m = 0;
    KMP_CUDA(&c, cudaMemcpyAsync(&m, &c.st->m, sizeof(m), cudaMemcpyDeviceToHost, c.stream), "read m");
    KMP_CUDA(&c, cudaStreamSynchronize(c.stream), "sync");
    int *changed = reinterpret_cast<int *>(c.partials + c.num_partials - 1);   // the last partial slot
    const int np = kmp::assign_num_partials(m, c.d);
    if (np + 1 > c.num_partials) return fail(&c, KMPAR_ERR_UNSUPPORTED, "candidate set larger than the point set");
    int cur = 0, t = 0;
    for (;; ++t) {
        KMP_CUDA(&c, cudaMemsetAsync(changed, 0, sizeof(int), c.stream), "memset changed");
        KMP_CUDA(&c, kmp::launch_assign(c.C, m, c.d, centers_dev, c.k, c.wl_lab[cur], t > 0 ? c.wl_lab[cur ^ 1] : nullptr,
                                        changed, c.partials, np, &c.st->argmin_fp64, c.stream),
                 "candidate assignment");
        int h = 0;
        KMP_CUDA(&c, cudaMemcpyAsync(&h, changed, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "read changed");
        KMP_CUDA(&c, cudaStreamSynchronize(c.stream), "sync");
        if (t > 0 && h == 0) break;
        if (t == max_iter) break;
        KMP_CUDA(&c, kmp::launch_weighted_centroids(c, m, c.wl_lab[cur], centers_dev), "weighted centroids");
        cur ^= 1;
    }
    if (iters) *iters = t;
    return KMPAR_OK;
}

// Each buffer is allocated once.  A call that failed part way (out of memory)
// leaves the buffers it got in place; the next call allocates the missing ones, and
// Lloyd runs only once all of them exist.
static kmpar_status ensure_lloyd_buffers(kmp::Ctx &c) {
    if (c.lloyd_ready) return KMPAR_OK;
    cudaError_t e;
#define KMP_ENSURE(ptr, count, what) \
    if (!(ptr) && (e = alloc(c, &(ptr), (count))) != cudaSuccess) return cuda_fail(&c, e, what)
    KMP_ENSURE(c.labels[0], (size_t)c.n, "alloc labels");
    KMP_ENSURE(c.labels[1], (size_t)c.n, "alloc labels");
    KMP_ENSURE(c.perm, (size_t)c.n, "alloc perm");
    KMP_ENSURE(c.hist, (size_t)c.nsb * c.k, "alloc hist");
    KMP_ENSURE(c.base, (size_t)c.k + 1, "alloc base");
    KMP_ENSURE(c.piece, (size_t)c.k + 1, "alloc pieces");
    KMP_ENSURE(c.chunk, (size_t)kmp::scan_chunks(c.nsb) * c.k, "alloc scan chunks");
    KMP_ENSURE(c.psum, (size_t)kmp::max_pieces(c.n, c.k) * c.d, "alloc piece sums");
    KMP_ENSURE(c.cost_dev, 4, "alloc cost");
    if (c.precision != KMPAR_FP32) KMP_ENSURE(c.dmin, (size_t)c.n, "alloc dmin");
    if (c.precision != KMPAR_FP32 && c.tc_cimg) {
        KMP_ENSURE(c.ll_ub, (size_t)c.n, "alloc Lloyd bounds");
        KMP_ENSURE(c.ll_lb, (size_t)c.n, "alloc Lloyd bounds");
        KMP_ENSURE(c.ll_rows, (size_t)c.n, "alloc Lloyd rows");
        KMP_ENSURE(c.ll_cnt, 1, "alloc Lloyd row count");
        KMP_ENSURE(c.ll_cold, (size_t)c.k * c.d, "alloc previous centers");
        KMP_ENSURE(c.ll_drift, (size_t)c.k, "alloc center drifts");
        KMP_ENSURE(c.ll_other, (size_t)c.k, "alloc center drifts");
    }
#undef KMP_ENSURE
    c.lloyd_ready = true;
    return KMPAR_OK;
}

kmpar_status kmpar_lloyd(kmpar_ctx *ctx, float *centers_dev, int32_t max_iter, int32_t *labels_dev,
                         int32_t *iters, double *final_cost, double *cost_hist) {
    if (!ctx) return fail(nullptr, KMPAR_ERR_ARG, "ctx is NULL");
    kmp::Ctx &c = ctx->c;
    if (!centers_dev) return fail(&c, KMPAR_ERR_ARG, "centers_dev is NULL");
    if (max_iter < 0) return fail(&c, KMPAR_ERR_ARG, "max_iter < 0");
    if (c.k > 49152) return fail(&c, KMPAR_ERR_UNSUPPORTED, "Lloyd supports k <= 49152");
    kmpar_status s = ensure_lloyd_buffers(c);
    if (s != KMPAR_OK) return s;
    // At a fixed point an iteration changes nothing (the same labels give the same
    // centroids bit for bit, and those the same labels), so the host reads the
    // per-iteration (cost, changed) records only every few iterations and stops at
    // the first one that changed no label; iterations run past it are no-ops.
    struct Rec { double cost; int changed; int pad; };
    static_assert(sizeof(Rec) == 16, "record layout");
    if (c.lloyd_rec_cap < max_iter + 1) {
        if (c.lloyd_rec) cudaFreeAsync(c.lloyd_rec, c.stream);
        c.lloyd_rec = nullptr;
        c.lloyd_rec_cap = 0;
        Rec *r = nullptr;
        KMP_CUDA(&c, alloc(c, &r, (size_t)(max_iter + 1)), "alloc Lloyd records");
        c.lloyd_rec = r;
        c.lloyd_rec_cap = max_iter + 1;
    }
    Rec *rec = reinterpret_cast<Rec *>(c.lloyd_rec);
    std::vector<Rec> hrec((size_t)max_iter + 1);
    int *changed = reinterpret_cast<int *>(c.cost_dev + 1);
    int cur = 0, t = 0, done = -1;
    // after the first assignment, rows whose bounds prove their center unchanged are
    // settled without the tensor pass (the results are the same)
    const bool bounded = kmp::lloyd_bounds_usable(c, centers_dev);
    auto keep_centers = [&]() -> cudaError_t {
        return bounded ? cudaMemcpyAsync(c.ll_cold, centers_dev, sizeof(float) * (size_t)c.k * c.d,
                                         cudaMemcpyDeviceToDevice, c.stream)
                       : cudaSuccess;
    };
    while (done < 0) {
        const int batch = t < 8 ? 4 : 8;
        const int t_end = std::min(max_iter, t + batch - 1);
        for (int tt = t; tt <= t_end; ++tt) {
            if (tt > t) {
                KMP_CUDA(&c, keep_centers(), "keep centers");
                KMP_CUDA(&c, kmp::launch_centroids(c, c.labels[cur], centers_dev), "centroid kernels");
                cur ^= 1;
            }
            KMP_CUDA(&c, cudaMemsetAsync(changed, 0, sizeof(int), c.stream), "memset changed");
            if (c.precision == KMPAR_FP32) {
                cudaEvent_t ev = nullptr;
                KMP_CUDA(&c, kmp::timing_begin(c, &ev), "timing");
                KMP_CUDA(&c, kmp::launch_assign(c.X, c.n, c.d, centers_dev, c.k, c.labels[cur],
                                                tt > 0 ? c.labels[cur ^ 1] : nullptr, changed, c.partials,
                                                c.num_partials, &c.st->argmin_fp64, c.stream),
                         "assign kernel");
                KMP_CUDA(&c, kmp::timing_end(c, ev, 1), "timing");
                KMP_CUDA(&c, kmp::launch_sum_f64(c.partials, c.num_partials, c.cost_dev, nullptr, c.stream),
                         "cost sum");
            } else if (bounded && tt > 0) {
                KMP_CUDA(&c, kmp::launch_lloyd_bounded_pass(c, centers_dev, c.labels[cur], c.labels[cur ^ 1],
                                                             changed, c.dmin),
                         "bounded assign pass");
                KMP_CUDA(&c, kmp::launch_sum_rows(c.dmin, c.n, c.partials, c.num_partials, c.cost_dev, nullptr,
                                                  c.stream),
                         "cost sum");
            } else {
                // after a centroid update, perm holds the rows sorted by their previous
                // label: the exact refine walks them in that order
                c.refine_order = tt > 0 ? c.perm : nullptr;
                const cudaError_t pe = kmp::launch_tc_pass(c, 0, centers_dev, c.k, c.labels[cur],
                                                           tt > 0 ? c.labels[cur ^ 1] : nullptr, changed, c.dmin, 1);
                c.refine_order = nullptr;
                KMP_CUDA(&c, pe, "tensor assign pass");
                KMP_CUDA(&c, kmp::launch_sum_rows(c.dmin, c.n, c.partials, c.num_partials, c.cost_dev, nullptr,
                                                  c.stream),
                         "cost sum");
            }
            KMP_CUDA(&c, cudaMemcpyAsync(rec + tt, c.cost_dev, sizeof(Rec), cudaMemcpyDeviceToDevice, c.stream),
                     "record");
        }
        KMP_CUDA(&c, cudaMemcpyAsync(hrec.data() + t, rec + t, sizeof(Rec) * (size_t)(t_end - t + 1),
                                     cudaMemcpyDeviceToHost, c.stream),
                 "read records");
        KMP_CUDA(&c, cudaStreamSynchronize(c.stream), "sync");
        KMP_CUDA(&c, kmp::timing_drain(c), "timing");
        if (c.tc_err) {
            kmpar_status ts = check_timeout(c);
            if (ts != KMPAR_OK) return ts;
        }
        for (int tt = t; tt <= t_end && done < 0; ++tt)
            if (tt > 0 && hrec[tt].changed == 0) done = tt;
        if (done < 0 && t_end == max_iter) done = max_iter;
        if (done < 0) {
            // the last iteration of the batch still needs its centroid update
            KMP_CUDA(&c, keep_centers(), "keep centers");
            KMP_CUDA(&c, kmp::launch_centroids(c, c.labels[cur], centers_dev), "centroid kernels");
            cur ^= 1;
            t = t_end + 1;
        }
    }
    t = done;
    const double cost = hrec[t].cost;
    if (cost_hist)
        for (int tt = 0; tt <= t; ++tt) cost_hist[tt] = hrec[tt].cost;
    if (labels_dev)
        KMP_CUDA(&c, cudaMemcpyAsync(labels_dev, c.labels[cur], sizeof(int32_t) * c.n, cudaMemcpyDeviceToDevice,
                                     c.stream), "copy labels");
    KMP_CUDA(&c, cudaStreamSynchronize(c.stream), "sync");
    c.lloyd_iters = t;
    if (iters) *iters = t;
    if (final_cost) *final_cost = cost;
    return KMPAR_OK;
}

kmpar_status kmpar_cost(const float *X, int64_t n, int32_t d, const float *C, int32_t k, int32_t precision,
                        double *phi, void *stream) {
    // every precision yields the same exact-FP32 cost; the CUDA-core pass computes it
    if (!X || !C || !phi) return fail(nullptr, KMPAR_ERR_ARG, "NULL pointer");
    if (n < 1 || n >= (int64_t)INT32_MAX || d < 1 || d > 4096 || k < 1)
        return fail(nullptr, KMPAR_ERR_ARG, "size out of range");
    if (!precision_supported(precision, d)) return fail(nullptr, KMPAR_ERR_UNSUPPORTED, "precision not built");
    cudaStream_t s = (cudaStream_t)stream;
    const int np = kmp::assign_num_partials(n, d);
    double *buf = nullptr;   // np partials, the sum, one counter
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&buf), sizeof(double) * (np + 2), s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "scratch alloc");
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(buf + np + 1);
    e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = kmp::launch_assign(X, n, d, C, k, nullptr, nullptr, nullptr, buf, np, cnt, s);
    if (e == cudaSuccess) e = kmp::launch_sum_f64(buf, np, buf + np, nullptr, s);
    double h = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, buf + np, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaFreeAsync(buf, s);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cost kernels");
    *phi = h;
    return KMPAR_OK;
}

kmpar_status kmpar_state(const kmpar_ctx *ctx, const float **D2_dev, const int32_t **idx_dev) {
    if (!ctx) return fail(nullptr, KMPAR_ERR_ARG, "ctx is NULL");
    if (D2_dev) *D2_dev = ctx->c.D2;
    if (idx_dev) *idx_dev = ctx->c.idx;
    return KMPAR_OK;
}

kmpar_status kmpar_get_stats(kmpar_ctx *ctx, kmpar_stats *out) {
    if (!ctx || !out) return fail(nullptr, KMPAR_ERR_ARG, "NULL pointer");
    kmp::Ctx &c = ctx->c;
    kmp::DevState st;
    KMP_CUDA(&c, cudaMemcpyAsync(&st, c.st, sizeof(st), cudaMemcpyDeviceToHost, c.stream), "read state");
    KMP_CUDA(&c, cudaStreamSynchronize(c.stream), "sync");
    memset(out, 0, sizeof(*out));
    out->n = c.n; out->m = st.m; out->d = c.d; out->k = c.k;
    out->rounds_done = c.rounds_done; out->lloyd_iters = c.lloyd_iters;
    for (int i = 0; i < kmp::kMaxRounds; ++i) out->round_added[i] = st.round_added[i];
    for (int i = 0; i <= kmp::kMaxRounds; ++i) out->phi[i] = st.phi_hist[i];
    out->sample_near = (int64_t)st.sample_near;
    out->sample_refined = (int64_t)st.sample_refined;
    out->argmin_fp64 = (int64_t)st.argmin_fp64;
    out->argmin_wide = (int64_t)st.argmin_wide;
    out->recluster_near = (int64_t)st.recluster_near;
    out->capacity_overflow = st.overflow;
    out->recluster_warn = st.warn;
    out->screen_rows = (int64_t)st.screen_rows;
    out->screen_fallback = (int64_t)st.screen_fallback;
    out->screen_exact = (int64_t)st.screen_exact;
    out->screen_listed = (int64_t)st.screen_listed;
    out->recluster_snapshots = (int64_t)st.recluster_snapshots;
    out->lloyd_settled = (int64_t)st.lloyd_settled;
    KMP_CUDA(&c, kmp::timing_drain(c), "timing");
    for (int i = 0; i < 2; ++i) {
        out->kernel_ms[i] = c.kernel_ms[i];
        out->kernel_launches[i] = c.kernel_launches[i];
    }
    return KMPAR_OK;
}

kmpar_status kmpar_uniforms(int64_t count, uint32_t round, uint32_t tag, uint64_t seed, double *out_dev,
                            void *stream) {
    if (count < 0 || (count > 0 && !out_dev)) return fail(nullptr, KMPAR_ERR_ARG, "bad arguments");
    if (count == 0) return KMPAR_OK;
    cudaError_t e = kmp::launch_uniforms(count, round, tag, seed, out_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "uniforms kernel");
    return KMPAR_OK;
}

kmpar_status kmpar_fit(const float *X, int64_t n, int32_t d, int32_t k, double ell, int32_t rounds, uint64_t seed,
                       int32_t precision, int32_t max_iter, float *centers_out, int32_t *labels_out,
                       double *seed_cost, double *final_cost, int32_t *iters, int32_t flags, void *stream) {
    if (!X || !centers_out) return fail(nullptr, KMPAR_ERR_ARG, "NULL pointer");
    if (n < 1 || d < 1 || k < 1) return fail(nullptr, KMPAR_ERR_ARG, "size out of range");
    cudaStream_t s = (cudaStream_t)stream;
    const bool host = (flags & KMPAR_HOST_BUFFERS) != 0;
    const float *Xd = X;
    float *Cd = centers_out;
    int32_t *Ld = labels_out;
    float *Xbuf = nullptr, *Cbuf = nullptr;   // device staging of the host buffers
    int32_t *Lbuf = nullptr;
    cudaError_t e = cudaSuccess;
    if (host) {
        e = cudaMallocAsync(reinterpret_cast<void **>(&Xbuf), sizeof(float) * (size_t)n * d, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(Xbuf, X, sizeof(float) * (size_t)n * d, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&Cbuf), sizeof(float) * (size_t)k * d, s);
        if (e == cudaSuccess && labels_out)
            e = cudaMallocAsync(reinterpret_cast<void **>(&Lbuf), sizeof(int32_t) * (size_t)n, s);
        if (e != cudaSuccess) {
            // hand back what the staging got before the failure
            if (Xbuf) cudaFreeAsync(Xbuf, s);
            if (Cbuf) cudaFreeAsync(Cbuf, s);
            if (Lbuf) cudaFreeAsync(Lbuf, s);
            return cuda_fail(nullptr, e, "fit staging");
        }
        Xd = Xbuf;
        Cd = Cbuf;
        Ld = Lbuf;
    }
    kmpar_ctx *ctx = nullptr;
    kmpar_status st = kmpar_init(&ctx, Xd, n, d, k, ell, rounds, seed, precision, stream);
    if (st == KMPAR_OK && (flags & KMPAR_EXACT_SAMPLING)) st = kmpar_set_sampling(ctx, KMPAR_SAMPLE_EXACT);
    if (st == KMPAR_OK && ((flags >> 16) & 0xFF)) st = kmpar_set_recluster(ctx, (flags >> 16) & 0xFF);
    for (int i = 1; st == KMPAR_OK && i <= rounds; ++i) st = kmpar_round(ctx, i, nullptr, nullptr);
    if (st == KMPAR_OK) st = kmpar_weight(ctx, nullptr, nullptr, nullptr);
    kmpar_status warn = KMPAR_OK;
    if (st == KMPAR_OK) {
        st = kmpar_recluster(ctx, Cd);
        if (st == KMPAR_WARN_FEW_CANDIDATES) { warn = st; st = KMPAR_OK; }
    }
    const int wl_iters = (flags >> 8) & 0xFF;
    if (st == KMPAR_OK && wl_iters > 0) st = kmpar_weighted_lloyd(ctx, Cd, wl_iters, nullptr);
    // Lloyd's first assignment is made with the seed centers: its cost is the seed cost
    std::vector<double> hist(max_iter >= 0 ? (size_t)max_iter + 1 : 1);
    if (st == KMPAR_OK) st = kmpar_lloyd(ctx, Cd, max_iter, Ld, iters, final_cost, hist.data());
    if (st == KMPAR_OK && seed_cost) *seed_cost = hist[0];
    if (st != KMPAR_OK && ctx) g_err = ctx->c.err;
    if (ctx) kmpar_destroy(ctx);
    if (host) {
        if (st == KMPAR_OK) {
            e = cudaMemcpyAsync(centers_out, Cd, sizeof(float) * (size_t)k * d, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && labels_out)
                e = cudaMemcpyAsync(labels_out, Ld, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s);
        }
        cudaFreeAsync(Xbuf, s);
        cudaFreeAsync(Cbuf, s);
        if (Lbuf) cudaFreeAsync(Lbuf, s);
        cudaError_t e2 = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = e2;
        if (st == KMPAR_OK && e != cudaSuccess) return cuda_fail(nullptr, e, "fit copy-out");
    }
    return st != KMPAR_OK ? st : warn;
}

kmpar_status kmpar_set_recluster(kmpar_ctx *ctx, int32_t batch) {
    if (!ctx) return fail(nullptr, KMPAR_ERR_ARG, "ctx is NULL");
    kmp::Ctx &c = ctx->c;
    if (batch < 0 || batch > kmp::kRsMaxBatch) return fail(&c, KMPAR_ERR_ARG, "recluster batch outside 0..64");
    c.rs_batch = batch;
    return KMPAR_OK;
}

kmpar_status kmpar_set_timing(kmpar_ctx *ctx, int32_t enable) {
    if (!ctx) return fail(nullptr, KMPAR_ERR_ARG, "ctx is NULL");
    ctx->c.timing = enable != 0;
    return KMPAR_OK;
}

int64_t kmpar_launch_count(void) { return (int64_t)kmp::g_launches.load(); }

kmpar_status kmpar_release_cached_memory(void) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (int dev = 0; dev < kMaxDevices; ++dev) {
        if (!g_pool[dev]) continue;
        const cudaError_t e = cudaMemPoolTrimTo(g_pool[dev], 0);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "release cached memory");
    }
    return KMPAR_OK;
}

void kmpar_destroy(kmpar_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->c.stream);
    for (auto &p : ctx->c.pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto ev : ctx->c.event_pool) cudaEventDestroy(ev);
    free_ctx(ctx->c);
    delete ctx;
}

}  // extern "C"
