// kmpar_internal.cuh -- context layout, device helpers and kernel launchers
// shared by the translation units of libkmpar (GB300, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/kmpar.h"
#include "nearest_tc.cuh"

namespace kmp {

constexpr uint32_t TAG_INIT = 1u;
constexpr uint32_t TAG_SAMPLE = 2u;
constexpr uint32_t TAG_RECLUSTER = 3u;

constexpr int kMaxRoundCap = 32768;   // single-CTA sort of one round's draws
constexpr int kMaxRounds = 64;

// Device-resident state of one context (one allocation, read by kernels).
struct DevState {
    int32_t m;              // candidates so far
    int32_t batch_begin;    // first candidate number of the last round's batch
    int32_t batch_cnt;      // size of the last round's batch
    int32_t drawn;          // atomic append counter of the current round
    int32_t overflow;       // capacity overflow flag
    int32_t warn;           // recluster ran out of mass
    int32_t changed;        // Lloyd: labels changed in the last assignment
    int32_t i0;             // first center
    double phi;             // current phi
    double phi_hist[kMaxRounds + 1];
    int32_t round_added[kMaxRounds];
    unsigned long long sample_near, sample_refined, argmin_fp64, argmin_wide, recluster_near;
    unsigned long long screen_rows, screen_fallback;   // tensor passes: rows screened, rows the pair screening left
    unsigned long long screen_exact;                   // rows that needed the exact scan
    unsigned long long screen_listed;                  // undecided round rows refined from the pass's own lists
    unsigned long long recluster_snapshots;            // batched reclustering: D^2 snapshots taken
    unsigned long long lloyd_settled;                  // Lloyd rows whose assignment the bounds settled
};

struct Ctx {
    // problem
    const float *X = nullptr;
    int64_t n = 0;
    int d = 0, k = 0, rounds = 0, precision = 0;
    double ell = 0;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    int dev = 0, num_sms = 0;
    // state machine
    int rounds_done = 0;
    bool weighted = false;
    int lloyd_iters = 0;
    // capacities
    int cap_round = 0, cap_total = 0;
    size_t alloc_bytes = 0;       // device memory this context holds
    // device buffers
    DevState *st = nullptr;
    float *D2 = nullptr;
    int32_t *idx = nullptr;
    int32_t *drawn = nullptr;     // cap_round
    int32_t *cand = nullptr;      // cap_total row numbers
    float *C = nullptr;           // cap_total x d candidate rows
    long long *w = nullptr;       // cap_total
    float *rD2 = nullptr;         // recluster D^2, 2 x cap_total rounded up to 32
    double *rc_cmass = nullptr;   // recluster chunk masses, 2 x ceil(cap_total / 32), then 2048 doubles of CTA slots
    float *rCT = nullptr;         // recluster grid form: candidates transposed (d x cap_total padded to 32)
    int32_t *wl_lab[2] = {nullptr, nullptr};   // weighted Lloyd: candidate labels (cap_total each)
    int rs_batch = 0;             // reclustering: 0 = one draw at a time, B = up to B draws per D^2 snapshot
    void *rs_buf = nullptr;       // batched reclustering: control word, proposals, their pair distances
    void *rc_sync = nullptr;      // recluster grid barrier / pick flag
    int *rc_err = nullptr;        // recluster timeout flag
    int32_t *chosen = nullptr;    // k
    double *partials = nullptr;   // per-block FP64 partial sums
    int num_partials = 0;
    // Lloyd
    int32_t *labels[2] = {nullptr, nullptr};
    int32_t *perm = nullptr;
    const int32_t *refine_order = nullptr;   // Lloyd: rows sorted by their previous label (perm), or null
    // Lloyd's bounds (tensor modes with the direct refine): per row an upper bound
    // of the distance to its center and a lower bound of the distance to every other
    // center (0: none); the centers before the last update, their drifts, the
    // largest drift of the other centers, and the rows the bounds leave open
    float *ll_ub = nullptr, *ll_lb = nullptr;
    float *ll_cold = nullptr, *ll_drift = nullptr, *ll_other = nullptr;
    int32_t *ll_rows = nullptr;
    int *ll_cnt = nullptr;
    int32_t *hist = nullptr;      // nsb x k
    int32_t *base = nullptr;      // k + 1
    int32_t *piece = nullptr;     // k + 1: first piece of each cluster
    int32_t *chunk = nullptr;     // column-scan chunk totals
    double *psum = nullptr;       // FP64 piece sums
    int nsb = 0, sort_block = 0;
    bool lloyd_ready = false;     // every Lloyd buffer below is allocated
    void *lloyd_rec = nullptr;    // per Lloyd iteration: (cost, labels changed), 16 bytes
    int lloyd_rec_cap = 0;
    double *cost_dev = nullptr;   // one FP64
    // tensor-core screening (BF16 and FP8 modes)
    int tc_fmt = -1;              // tc::Fmt of the screening operands
    bool tc_list = false;         // undecided rows get the list pass before the exact scan
    uint8_t *tc_img = nullptr;    // swizzled center tiles
    uint8_t *tc_ximg = nullptr;   // swizzled BF16 image of X (built once per context)
    float *tc_xnorm = nullptr;    // ||x'||^2 per point (x' = x - anchor)
    float *tc_anchor = nullptr;   // d column means of X
    double *tc_anchor_part = nullptr;   // per-block column sums behind the anchor
    unsigned int *tc_cmax = nullptr;
    int *tc_err = nullptr;        // first timeout code of a tensor pass
    int32_t *cand1 = nullptr;     // per row: first center of the best screened pair of the last tensor pass, or -1
    float *tc_v2 = nullptr;       // per row: smallest screened value outside that pair
    int32_t *fix_rows = nullptr;  // rows left to the exact CUDA-core pass
    int *fix_cnt = nullptr;
    float *dmin = nullptr;        // Lloyd: exact d^2 of each point's chosen center
    float *tc_ncol = nullptr;     // norms in the epilogue: ||c'||^2 per pass-local center
    float *tc_tscale = nullptr;   // per center tile scale
    float *tc_xscale = nullptr;   // FP8: per-row scale of the points image
    float *tc_ub = nullptr;       // per row: exact upper bound of the deciding distance (undecided rows)
    uint8_t *tc_cimg = nullptr;   // list pass: image rows of the undecided rows, compacted
    float *tc_cscale = nullptr;   // list pass: their scales
    float *tc_thr = nullptr;      // list pass: their thresholds
    int32_t *tc_lst = nullptr;    // list pass: 4 x kListSlots centers per row
    int32_t *tc_lcnt = nullptr;   // list pass: entries per row and column group
    int32_t *fix_rows2 = nullptr; // rows left to the exact scan after the list pass
    int *fix_cnt2 = nullptr;
    // exactly-l rounds (Sec. 5.3): 0 = independent draws, 1 = floor(l) per round
    int sampling = 0;
    uint32_t *ex_keys = nullptr;  // per point: FP32 clock bits
    void *ex_ws = nullptr;        // radix-select state
    int32_t *ex_ties = nullptr;   // points whose clock equals the last drawn one
    // CUDA-event timing of the distance passes (0 = rounds, 1 = Lloyd assign)
    bool timing = false;
    struct Pending { cudaEvent_t a, b; int cls; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    double kernel_ms[2] = {0, 0};
    int64_t kernel_launches[2] = {0, 0};
    std::string err;
};

// process-wide count of kernel launches made by this library
extern std::atomic<long long> g_launches;
inline void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// exactly-l rounds (exact_sample.cu)
size_t exact_work_bytes();
int exact_tie_cap();
cudaError_t launch_sample_exact(Ctx &c, int round);

// timing helpers (no-ops unless c.timing)
cudaError_t timing_begin(Ctx &c, cudaEvent_t *a);
cudaError_t timing_end(Ctx &c, cudaEvent_t a, int cls);
cudaError_t timing_drain(Ctx &c);   // call after a stream synchronisation

// ---------------------------------------------------------------- device helpers

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplies with the published multipliers; key bumped by the Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = c0 * 0xD2511F53u, hi0 = __umulhi(c0, 0xD2511F53u);
        const uint32_t lo1 = c2 * 0xCD9E8D57u, hi1 = __umulhi(c2, 0xCD9E8D57u);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// uniform double in [0,1) from counter (i, round, tag), key = seed: (a 2^26 + b) 2^-53
__device__ __forceinline__ double uniform53(uint64_t i, uint32_t round, uint32_t tag, uint64_t seed) {
    const uint4 w = philox4x32_10((uint32_t)i, (uint32_t)(i >> 32), round, tag, (uint32_t)seed,
                                  (uint32_t)(seed >> 32));
    const double a = (double)(w.x >> 5), b = (double)(w.y >> 6);
    return __dmul_rn(__dadd_rn(__dmul_rn(a, 67108864.0), b), 1.0 / 9007199254740992.0);
}

// ||x - c||^2 in FP64, difference form, ascending coordinates, separate rounded
// multiply and add (the definition, Sec. 3.1).
__device__ __forceinline__ double dist2_fp64(const float *__restrict__ x, const float *__restrict__ c, int d) {
    double s = 0.0;
    for (int q = 0; q < d; ++q) {
        const double t = __dsub_rn((double)x[q], (double)c[q]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

// ||x - c||^2 in FP32, difference form: t = x_q - c_q rounded, acc = fma(t, t, acc)
// for q ascending.  This is THE FP32 distance of the library: every precision mode
// stores this value.
__device__ __forceinline__ float dist2_fp32(const float *__restrict__ x, const float *__restrict__ c, int d) {
    float s = 0.f;
    for (int q = 0; q < d; ++q) {
        const float t = __fsub_rn(x[q], c[q]);
        s = __fmaf_rn(t, t, s);
    }
    return s;
}

// Relative window inside which two FP32 distances may be ordered differently from
// their FP64 values: each carries at most (d+1) 2^-24 relative error (sum of d
// non-negative terms), so twice that plus slack.
__host__ __device__ __forceinline__ float fp32_tie_window(int d) {
    return (float)(2 * d + 8) * 5.9604645e-8f;
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_sum_i32(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum of one FP64 per thread (fixed shuffle tree, then warps in
// order).  Result valid in thread 0.  blockDim.x must be a multiple of 32, <= 1024.
__device__ __forceinline__ double block_sum_f64(double v, double *sh /*32*/) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum_f64(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int i = 0; i < nw; ++i) r += sh[i];
    }
    return r;
}

// ---------------------------------------------------------------- launchers
// (each returns cudaGetLastError() of its launch)
cudaError_t launch_init_first(Ctx &c);
cudaError_t launch_round(Ctx &c, int round);
cudaError_t launch_round_distance(Ctx &c, int round);
cudaError_t launch_phi_finalize(Ctx &c, int nparts, double *out, double *hist_slot);
cudaError_t launch_weights(Ctx &c);
cudaError_t launch_recluster(Ctx &c, float *centers);
// batched reclustering (recluster_batch.cu): up to kRsMaxBatch draws per D^2 snapshot
constexpr int kRsMaxBatch = 64;
constexpr int kRsMaxProposals = 2 * kRsMaxBatch;
size_t recluster_batch_bytes();
cudaError_t launch_recluster_batch(Ctx &c, float *centers);
cudaError_t launch_transpose_cand(Ctx &c);   // candidates -> c.rCT (d x cap_total padded to 32)
size_t recluster_sync_bytes();
size_t recluster_grid_floats(const Ctx &c);   // floats of the transposed copy the grid form needs (0: none)
cudaError_t launch_weighted_centroids(const Ctx &c, int m, const int32_t *lab, float *centers);
cudaError_t launch_assign(const float *X, int64_t n, int d, const float *C, int k, int32_t *labels,
                          const int32_t *prev, int *changed, double *partials, int nparts,
                          unsigned long long *fp64_cnt, cudaStream_t s);
int assign_num_partials(int64_t n, int d);
cudaError_t launch_centroids(Ctx &c, const int32_t *labels, float *centers);
int sort_block_size(int64_t n, int k);
int64_t max_pieces(int64_t n, int k);
int64_t scan_chunks(int nsb);
cudaError_t count_fixups(Ctx &c, const int *exact_cnt);   // adds the pass's counts to the screening stats
cudaError_t launch_tc_pass(Ctx &c, int mode_round, const float *C, int k, int32_t *labels, const int32_t *prev,
                           int *changed, float *dmin, int timing_cls, const int32_t *rows = nullptr,
                           const int *rows_cnt = nullptr);
// Lloyd's bounds (round_simt.cu): whether this context can use them with centers C,
// and one assignment after a centroid update that uses them
bool lloyd_bounds_usable(const Ctx &c, const float *C);
cudaError_t launch_lloyd_bounded_pass(Ctx &c, const float *C, int32_t *labels, const int32_t *prev, int *changed,
                                      float *dmin);
cudaError_t launch_sum_rows(const float *v, int64_t n, double *partials, int max_parts, double *out, double *copy,
                            cudaStream_t s);
cudaError_t launch_uniforms(int64_t count, uint32_t round, uint32_t tag, uint64_t seed, double *out,
                            cudaStream_t s);
cudaError_t launch_sum_f64(const double *parts, int nparts, double *out, double *copy, cudaStream_t s);

}  // namespace kmp
