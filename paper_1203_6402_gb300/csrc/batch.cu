// batch.cu -- many independent k-means|| problems in one call (kmpar_batch_run):
// Algorithm 2 (Sec. 3.3) and Lloyd's iteration (Sec. 1, Sec. 3.1) per problem,
// one thread block per problem, every step on the device.  The data-parallel
// pattern of Sec. 3.5 is applied across problems: a block owns its problem from
// the first center to the last centroid update, so no grid-wide synchronisation
// is needed and the blocks run in any order (largest problems first).
//
// Per problem (kBT threads, the point loop in chunks of kBT rows, thread = row,
// the row's coordinates in registers, centers in kBTile-row shared-memory tiles):
//   init     i0 = floor(u n), D^2 = ||x - x_i0||^2, idx = 0, phi = sum D^2 (FP64)
//   round i  every x drawn with p = min(1, l D^2 / phi) (Philox, FP64 re-decision
//            of near draws), appended in ascending point order by an ordered
//            block compaction (no sort); D^2/idx against the batch
//   step 7   w_c = #{x : idx(x) = c} (shared-memory integer atomics)
//   step 8   weighted k-means++: per draw a blocked FP64 prefix over the masses,
//            the first candidate whose prefix exceeds u * total
//   Lloyd    assignment with the FP32 path's decision rule; centroids from a
//            stable counting sort by label (warp-private label counters,
//            __match_any_sync ranks) and compensated FP32 sums in ascending
//            point order, divided in FP64, rounded to FP32 once
// Distances are the exact FP32 difference form (ascending coordinates, one
// rounded subtraction and one FMA each), so every decision equals kmpar_fit's
// FP32 path on the same problem.
#include <float.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <vector>

#include <cooperative_groups.h>

#include "kmpar_internal.cuh"

namespace cg = cooperative_groups;

namespace kmp {
void set_thread_error(const std::string &m);

namespace {

constexpr int kBT = 256;          // threads per problem block
constexpr int kBW = kBT / 32;     // warps per block
constexpr int kBTile = 32;        // centers per shared-memory tile
constexpr int kBMaxK = 512;
constexpr int kBMaxRounds = 16;
constexpr int kBMaxCap = 4096;    // per-round draw capacity

// device copy of one problem with its work-space offsets
struct BProb {
    int64_t x_off, n;
    int d, k;
    double ell;
    int rounds, max_iter;
    uint64_t seed;
    int64_t c_off, l_off, cand_off;   // outputs
    int64_t p_off, m_off;             // work space: per-point arrays, per-candidate arrays
    int cap_round, cap_total;
};

struct BRes {
    long long m;
    double seed_cost, final_cost;
    int iters, status;
    unsigned long long sample_near, argmin_fp64, recluster_near;
};

struct BArgs {
    const float *X;
    const BProb *probs;
    const int32_t *order;    // problems of this launch, largest first
    float *centers;
    int32_t *labels_out;     // nullable
    int32_t *cand_out;       // nullable
    long long *w_out;        // nullable
    BRes *res;
    // work space
    float *D2;
    int32_t *idx, *lab, *perm;
    int32_t *cand;
    int32_t *w;
    float *rD2;
};

enum { BM_FIRST = 0, BM_ROUND = 1, BM_ASSIGN = 2 };

// Deterministic block sum of one FP64 per thread: fixed shuffle tree, warps in
// order; the result is returned to every thread.
__device__ __forceinline__ double bsum_f64(double v, double *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    for (int i = 0; i < kBW; ++i) r += sh[i];
    return r;
}

__device__ __forceinline__ int bsum_i32(int v, int *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int r = 0;
    for (int i = 0; i < kBW; ++i) r += sh[i];
    return r;
}

// one term of the exact FP32 difference form: t = x - c rounded, a = fma(t, t, a)
__device__ __forceinline__ void sq_acc(float x, float c, float &a) {
    const float t = __fsub_rn(x, c);
    a = __fmaf_rn(t, t, a);
}

__device__ __forceinline__ void take_better(double v, int j, double &best, int &bj) {
    if (v < best || (v == best && j < bj)) { best = v; bj = j; }
}

// Shared state of one block.
template <int DP>
struct BShared {
    float tile[kBTile * DP];
    double red[kBW];
    int redi[kBW];
    int hist[kBW][kBMaxK];     // Lloyd: per-warp label counts, then the warps' running bases
    int base[kBMaxK + 1];      // step 8: the chosen candidates; Lloyd: cluster offsets
    int wpos[kBW];
    int s_int[4];
    int wl_tot[kBMaxK];        // Lloyd (rank 0): label totals over the cluster
    double s_dslot;
    int s_islot;
    unsigned long long s_uslot;
    unsigned long long s_near, s_fp64, s_rnear;
};

// One pass over the rows [r0, r1) of a problem against `cnt` centers: the rows of C_rows (a
// center matrix, stride d) or, when cand is given, X rows cand[begin + r].  Each
// thread holds one row's coordinates in registers (padded to DP with zeros: they
// add exact zeros to the sums) and keeps the lexicographic (value, center number)
// top-2 over centers in ascending order; the decision is the FP32 path's:
//   FIRST   D^2 = the single distance, idx = 0
//   ROUND   the current center is replaced by the best new one when nearer; two
//           or more of (current, best, runner-up) within the FP32 tie window are
//           re-decided in FP64 (difference form, no FMA), equal values keeping
//           the lower center number
//   ASSIGN  the best, re-decided in FP64 against the runner-up inside the window
// Returns the block's FP64 sum of the stored distances (D^2 or the chosen
// center's distance) and sets *changed to the block's number of changed labels.
template <int DP, int MODE>
__device__ double dist_pass(BShared<DP> &sh, const float *__restrict__ Xp, int64_t r0, int64_t r1, int d,
                            const float *__restrict__ C_rows, const int32_t *__restrict__ cand, int begin, int cnt,
                            float *D2, int32_t *idx, int32_t *lab, int *changed, unsigned long long *fp64_cnt) {
    const int tid = threadIdx.x;
    const float W = fp32_tie_window(d);
    double acc_sum = 0.0;
    int chg = 0;
    unsigned long long nfp64 = 0;
    for (int64_t base = r0; base < r1; base += kBT) {
        const int64_t pt = base + tid;
        const bool valid = pt < r1;
        const float *xrow = Xp + (valid ? pt : 0) * (int64_t)d;
        float xr[DP];
#pragma unroll
        for (int q = 0; q < DP; ++q) xr[q] = (valid && q < d) ? __ldg(xrow + q) : 0.f;
        float b1 = FLT_MAX, b2 = FLT_MAX;
        int i1 = -1, i2 = -1;
        for (int t0 = 0; t0 < cnt; t0 += kBTile) {
            const int nt = min(kBTile, cnt - t0);
            __syncthreads();
            for (int e = tid; e < kBTile * DP; e += kBT) {
                const int r = e / DP, q = e - r * DP;
                float v = 0.f;
                if (r < nt && q < d) {
                    const int j = begin + t0 + r;
                    const float *row = cand ? Xp + (int64_t)cand[j] * d : C_rows + (int64_t)j * d;
                    v = __ldg(row + q);
                }
                sh.tile[e] = v;
            }
            __syncthreads();
            if (valid) {
                int r = 0;
                // NCH independent chains (one per center) interleaved per coordinate
                constexpr int NCH = 8;
                for (; r + NCH <= nt; r += NCH) {
                    float acc[NCH];
#pragma unroll
                    for (int u = 0; u < NCH; ++u) acc[u] = 0.f;
#pragma unroll
                    for (int q4 = 0; q4 < DP / 4; ++q4) {
                        float4 cv[NCH];
#pragma unroll
                        for (int u = 0; u < NCH; ++u) cv[u] = reinterpret_cast<const float4 *>(sh.tile + (r + u) * DP)[q4];
#pragma unroll
                        for (int u = 0; u < NCH; ++u) sq_acc(xr[4 * q4 + 0], cv[u].x, acc[u]);
#pragma unroll
                        for (int u = 0; u < NCH; ++u) sq_acc(xr[4 * q4 + 1], cv[u].y, acc[u]);
#pragma unroll
                        for (int u = 0; u < NCH; ++u) sq_acc(xr[4 * q4 + 2], cv[u].z, acc[u]);
#pragma unroll
                        for (int u = 0; u < NCH; ++u) sq_acc(xr[4 * q4 + 3], cv[u].w, acc[u]);
                    }
#pragma unroll
                    for (int u = 0; u < NCH; ++u) {
                        const int j = begin + t0 + r + u;
                        const float a = acc[u];
                        if (a < b2) {
                            if (a < b1) { b2 = b1; i2 = i1; b1 = a; i1 = j; }
                            else { b2 = a; i2 = j; }
                        }
                    }
                }
                for (; r < nt; ++r) {
                    float a = 0.f;
                    const float4 *c4 = reinterpret_cast<const float4 *>(sh.tile + r * DP);
#pragma unroll
                    for (int q4 = 0; q4 < DP / 4; ++q4) {
                        const float4 u = c4[q4];
                        sq_acc(xr[4 * q4 + 0], u.x, a);
                        sq_acc(xr[4 * q4 + 1], u.y, a);
                        sq_acc(xr[4 * q4 + 2], u.z, a);
                        sq_acc(xr[4 * q4 + 3], u.w, a);
                    }
                    const int j = begin + t0 + r;
                    if (a < b2) {
                        if (a < b1) { b2 = b1; i2 = i1; b1 = a; i1 = j; }
                        else { b2 = a; i2 = j; }
                    }
                }
            }
        }
        if (!valid) continue;
        auto crow = [&](int j) -> const float * {
            return cand ? Xp + (int64_t)cand[j] * d : C_rows + (int64_t)j * d;
        };
        float stored = 0.f;
        if (MODE == BM_FIRST) {
            stored = (i1 >= 0) ? b1 : __int_as_float(0x7f800000);
            D2[pt] = stored;
            idx[pt] = 0;
        } else if (MODE == BM_ASSIGN) {
            int l = i1 >= 0 ? i1 : 0;
            stored = b1;
            if (i2 >= 0 && b2 <= b1 + W * b1) {
                double best = dist2_fp64(xrow, crow(i1), d);
                int bj = i1;
                take_better(dist2_fp64(xrow, crow(i2), d), i2, best, bj);
                if (bj == i2) { l = i2; stored = b2; }
                ++nfp64;
            }
            if (changed) chg += (lab[pt] != l);
            lab[pt] = l;
        } else {
            const float old = D2[pt];
            const int oi = idx[pt];
            const float m32 = fminf(old, b1);
            const float lim = m32 + W * m32;
            const bool in_old = (oi >= 0) && old <= lim;
            const bool in1 = i1 >= 0 && b1 <= lim;
            const bool in2 = i2 >= 0 && b2 <= lim;
            int win = -1;
            float wv = old;
            if ((int)in_old + (int)in1 + (int)in2 >= 2) {
                double best = DBL_MAX;
                int bj = INT_MAX;
                if (in_old) take_better(dist2_fp64(xrow, Xp + (int64_t)cand[oi] * d, d), oi, best, bj);
                if (in1) take_better(dist2_fp64(xrow, crow(i1), d), i1, best, bj);
                if (in2) take_better(dist2_fp64(xrow, crow(i2), d), i2, best, bj);
                ++nfp64;
                if (bj == i1) { win = i1; wv = b1; }
                else if (bj == i2) { win = i2; wv = b2; }
            } else if (i1 >= 0 && b1 < old) {
                win = i1; wv = b1;
            }
            if (win >= 0) { D2[pt] = wv; idx[pt] = win; stored = wv; }
            else stored = old;
        }
        acc_sum += (double)stored;
    }
    if (nfp64) atomicAdd(fp64_cnt, nfp64);
    if (MODE == BM_ASSIGN && changed) *changed = bsum_i32(chg, sh.redi);   // every thread
    return bsum_f64(acc_sum, sh.red);
}

// Block-wide exclusive prefix of one FP64 per thread in thread order (warp scans,
// then the warp totals in order); returns the thread's exclusive prefix and the
// total (to every thread).
__device__ __forceinline__ double bscan_f64(double v, double *sh, double *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = incl;
    __syncthreads();
    double before = 0.0, tot = 0.0;
    for (int i = 0; i < kBW; ++i) {
        if (i < wid) before += sh[i];
        tot += sh[i];
    }
    *total = tot;
    double excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0.0;
    return before + excl;
}

__device__ __forceinline__ int bmin_i32(int v, int *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int r = INT_MAX;
    for (int i = 0; i < kBW; ++i) r = min(r, sh[i]);
    return r;
}

__device__ __forceinline__ int bmax_i32(int v, int *sh) { return -bmin_i32(-v, sh); }

// ---- a problem split over a thread-block cluster of CS blocks (CS = 1: one block)
// Barrier of the cluster (hardware; its arrive/wait pair orders memory at cluster
// scope, and the fence makes the global writes of this block visible first).
template <int CS>
__device__ __forceinline__ void csync() {
    if (CS > 1) {
        __threadfence();
        cg::this_cluster().sync();
    } else {
        __syncthreads();
    }
}

// Sum over the cluster's blocks, in rank order, of a block-uniform value: every
// block gets the same result.
template <int CS, typename T>
__device__ __forceinline__ T csum(T v, T *slot) {
    if (CS == 1) return v;
    __syncthreads();
    if (threadIdx.x == 0) *slot = v;
    cg::this_cluster().sync();
    T r = 0;
    for (int q = 0; q < CS; ++q) r += *cg::this_cluster().map_shared_rank(slot, q);
    cg::this_cluster().sync();   // no block overwrites its slot before every block has read it
    return r;
}

// Exclusive prefix in rank order and total of a block-uniform count.
template <int CS>
__device__ __forceinline__ int cprefix(int v, int *slot, int *total) {
    if (CS == 1) { *total = v; return 0; }
    __syncthreads();
    if (threadIdx.x == 0) *slot = v;
    cg::this_cluster().sync();
    const int me = (int)cg::this_cluster().block_rank();
    int before = 0, tot = 0;
    for (int q = 0; q < CS; ++q) {
        const int c = *cg::this_cluster().map_shared_rank(slot, q);
        if (q < me) before += c;
        tot += c;
    }
    cg::this_cluster().sync();
    *total = tot;
    return before;
}

// Knuth's TwoSum: (s, c) += x with s the rounded sum and c the accumulated
// rounding errors (all FP32, each operation rounded to nearest)
__device__ __forceinline__ void two_sum_add(float &s, float &c, float x) {
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    c = __fadd_rn(c, e);
    s = t;
}

// One problem per cluster of CS blocks (CS = 1: one block).  Block rank r of the
// cluster owns the contiguous rows [r0, r1); every per-point step runs on the
// block's own rows, and the cluster combines in rank order: phi and the Lloyd
// cost and change counts (sums), the round draws (each block appends its draws in
// ascending point order after those of the lower ranks), and Lloyd's counting sort
// (label offsets over (rank, warp) in order).  Step 8 runs in rank 0.
template <int DP, int CS>
__global__ void __launch_bounds__(kBT, DP == 128 ? 1 : 2) batch_kernel(BArgs a, int first) {
    __shared__ BShared<DP> sh;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int rank = CS > 1 ? (int)cg::this_cluster().block_rank() : 0;
    const int pi = a.order[first + blockIdx.x / CS];
    const BProb P = a.probs[pi];
    const float *X = a.X + P.x_off;
    const int64_t n = P.n;
    const int d = P.d, k = P.k;
    const int64_t per = (n + CS - 1) / CS;
    const int64_t r0 = min(n, (int64_t)rank * per), r1 = min(n, r0 + per);
    float *D2 = a.D2 + P.p_off;
    int32_t *idx = a.idx + P.p_off, *lab = a.lab + P.p_off, *perm = a.perm + P.p_off;
    int32_t *cand = a.cand + P.m_off, *w = a.w + P.m_off;
    float *rD2 = a.rD2 + P.m_off;
    float *C = a.centers + P.c_off;
    if (tid == 0) {
        sh.s_near = 0; sh.s_fp64 = 0; sh.s_rnear = 0;
        if (rank == 0) {
            // Alg. 2 step 1: the first center, uniform over the problem's points
            const double u = uniform53(0, 0, TAG_INIT, P.seed);
            int64_t i0 = (int64_t)floor(__dmul_rn(u, (double)n));
            if (i0 >= n) i0 = n - 1;
            cand[0] = (int32_t)i0;
        }
    }
    csync<CS>();
    // step 2: D^2 to the first center and psi
    double phi = csum<CS>(dist_pass<DP, BM_FIRST>(sh, X, r0, r1, d, nullptr, cand, 0, 1, D2, idx, nullptr, nullptr,
                                                  &sh.s_fp64),
                          &sh.s_dslot);
    int m = 1, status = KMPAR_OK;
    for (int r = 1; r <= P.rounds; ++r) {
        // step 4: independent draws of the block's rows; p and the near-draw rule as
        // in the single-problem path
        auto draw = [&](int64_t pt, bool &take, unsigned long long &near) {
            const float dd = D2[pt];
            double pr = 0.0;
            if (phi > 0.0) pr = fmin(1.0, __ddiv_rn(__dmul_rn(P.ell, (double)dd), phi));
            const double u = uniform53((uint64_t)pt, (uint32_t)r, TAG_SAMPLE, P.seed);
            if (dd > 0.f && fabs(u - pr) <= 1e-5) {
                // the FP32 D^2 could decide this draw: use the FP64 distance of the definition
                const double d64 = dist2_fp64(X + pt * d, X + (int64_t)cand[idx[pt]] * d, d);
                pr = fmin(1.0, __ddiv_rn(__dmul_rn(P.ell, d64), phi));
            }
            if (fabs(u - pr) <= 1e-6) ++near;
            take = u < pr;
        };
        // the block's place among the cluster's draws (a counting pass first)
        int mine = 0;
        if (CS > 1) {
            unsigned long long dummy = 0;
            int cntl = 0;
            for (int64_t pt = r0 + tid; pt < r1; pt += kBT) {
                bool take;
                draw(pt, take, dummy);
                cntl += take;
            }
            mine = bsum_i32(cntl, sh.redi);
        }
        int appended_all = 0;
        const int before_blocks = cprefix<CS>(mine, &sh.s_islot, &appended_all);
        int appended = 0;
        unsigned long long near = 0;
        for (int64_t base = r0; base < r1; base += kBT) {
            const int64_t pt = base + tid;
            bool take = false;
            if (pt < r1) draw(pt, take, near);
            const unsigned mask = __ballot_sync(0xffffffffu, take);
            if (lane == 0) sh.wpos[wid] = __popc(mask);
            __syncthreads();
            int before = 0, tot = 0;
            for (int i = 0; i < kBW; ++i) {
                if (i < wid) before += sh.wpos[i];
                tot += sh.wpos[i];
            }
            if (take) {
                const int pos = before_blocks + appended + before + __popc(mask & ((1u << lane) - 1u));
                if (pos < P.cap_round) cand[m + pos] = (int32_t)pt;
            }
            appended += tot;
            __syncthreads();   // wpos is rewritten by the next chunk
        }
        if (near) atomicAdd(&sh.s_near, near);
        if (CS == 1) appended_all = appended;
        if (appended_all > P.cap_round) { status = KMPAR_ERR_CAPACITY; break; }
        csync<CS>();           // the batch's row numbers are visible to the whole cluster
        // step 5: D^2 and idx against the batch, then phi
        phi = csum<CS>(dist_pass<DP, BM_ROUND>(sh, X, r0, r1, d, nullptr, cand, m, appended_all, D2, idx, nullptr,
                                               nullptr, &sh.s_fp64),
                       &sh.s_dslot);
        m += appended_all;
    }
    BRes res{};
    res.m = m;
    if (status == KMPAR_OK) {
        // step 7: weights
        for (int j = (int)(rank * kBT) + tid; j < m; j += CS * kBT) w[j] = 0;
        csync<CS>();
        for (int64_t pt = r0 + tid; pt < r1; pt += kBT) atomicAdd(&w[idx[pt]], 1);
        csync<CS>();
        // step 8 (rank 0): weighted k-means++ over the m candidates
        bool warn = false;
        if (rank == 0) {
            const int q = (m + kBT - 1) / kBT;
            const int lo = min(m, tid * q), hi = min(m, lo + q);
            int *chosen = sh.base;
            for (int t = 0; t < k; ++t) {
                double local = 0.0;
                for (int j = lo; j < hi; ++j)
                    local += t == 0 ? (double)w[j] : __dmul_rn((double)w[j], (double)rD2[j]);
                double total;
                const double excl = bscan_f64(local, sh.red, &total);
                if (!(total > 0.0)) {
                    // positive mass exhausted: the remaining centers repeat the first chosen one
                    const int src = t > 0 ? chosen[0] : 0;
                    for (int s2 = t; s2 < k; ++s2) {
                        for (int qq = tid; qq < d; qq += kBT)
                            C[(int64_t)s2 * d + qq] = X[(int64_t)cand[src] * d + qq];
                        if (tid == 0) chosen[s2] = src;
                    }
                    warn = true;
                    break;
                }
                const double target = __dmul_rn(uniform53((uint64_t)t, 0, TAG_RECLUSTER, P.seed), total);
                int hit = INT_MAX;
                double cum0 = 0.0, cum = 0.0, run = excl;
                for (int j = lo; j < hi; ++j) {
                    const double e = t == 0 ? (double)w[j] : __dmul_rn((double)w[j], (double)rD2[j]);
                    const double pre = run;
                    run = run + e;
                    if (run > target) { hit = j; cum0 = pre; cum = run; break; }
                }
                int pick = bmin_i32(hit, sh.redi);
                if (pick == INT_MAX) {
                    // the target rounded past every prefix: the last candidate with positive mass
                    int lastp = -1;
                    for (int j = lo; j < hi; ++j)
                        if ((t == 0 ? (double)w[j] : __dmul_rn((double)w[j], (double)rD2[j])) > 0.0) lastp = j;
                    pick = bmax_i32(lastp, sh.redi);
                    if (tid == 0) atomicAdd(&sh.s_rnear, 1ull);
                } else if (hit == pick &&
                           (fabs(target - cum0) <= 1e-6 * total || fabs(cum - target) <= 1e-6 * total)) {
                    atomicAdd(&sh.s_rnear, 1ull);
                }
                if (tid == 0) chosen[t] = pick;
                const float *prow = X + (int64_t)cand[pick] * d;
                for (int qq = tid; qq < DP; qq += kBT) {
                    const float v = qq < d ? prow[qq] : 0.f;
                    sh.tile[qq] = v;   // the pick's row, zero-padded to DP
                    if (qq < d) C[(int64_t)t * d + qq] = v;
                }
                __syncthreads();
                // D^2 of every candidate to the centers drawn so far, in the exact FP32
                // chain (t = x_q - c_q, fma, q ascending; padded zeros add 0), 16
                // coordinates at a time loaded into registers together.  The partial
                // sums never decrease, so once one reaches the candidate's D^2 the rest
                // cannot lower it and is skipped (most candidates are far from the pick).
                for (int j = tid; j < m; j += kBT) {
                    const float *xj = X + (int64_t)cand[j] * d;
                    const float lim = t == 0 ? __uint_as_float(0x7f800000u) : rD2[j];
                    float v = 0.f;
#pragma unroll
                    for (int q0 = 0; q0 < DP; q0 += 16) {
                        float xr[16];
#pragma unroll
                        for (int u = 0; u < 16; ++u) xr[u] = q0 + u < d ? __ldg(xj + q0 + u) : 0.f;
#pragma unroll
                        for (int u = 0; u < 16; ++u) sq_acc(xr[u], sh.tile[q0 + u], v);
                        if (v >= lim) break;
                    }
                    if (v < lim) rD2[j] = v;
                }
                __syncthreads();
            }
        }
        if (warn) status = KMPAR_WARN_FEW_CANDIDATES;
        csync<CS>();           // the seed centers are visible to the whole cluster
        // Lloyd's iteration from the seed centers
        int it = 0;
        double cost = 0.0;
        for (;; ++it) {
            int chg = 0;
            const double part = dist_pass<DP, BM_ASSIGN>(sh, X, r0, r1, d, C, nullptr, 0, k, nullptr, nullptr, lab,
                                                         it > 0 ? &chg : nullptr, &sh.s_fp64);
            cost = csum<CS>(part, &sh.s_dslot);
            if (it > 0) chg = csum<CS>(chg, &sh.s_islot);
            if (it == 0) res.seed_cost = cost;
            if (it > 0 && chg == 0) break;
            if (it == P.max_iter) break;
            // stable counting sort by label: warp wr of block r owns the contiguous rows
            // [r0 + wr npw, r0 + (wr+1) npw); offsets run over (rank, warp) in order
            const int64_t npw = (r1 - r0 + kBW - 1) / kBW;
            const int64_t w0 = min(r1, r0 + (int64_t)wid * npw), w1 = min(r1, w0 + npw);
            for (int l = tid; l < kBW * kBMaxK; l += kBT) (&sh.hist[0][0])[l] = 0;
            __syncthreads();
            for (int64_t c0 = w0; c0 < w1; c0 += 32) {
                const int64_t pt = c0 + lane;
                const int l = pt < w1 ? lab[pt] : -1;
                const unsigned peers = __match_any_sync(0xffffffffu, l);
                if (l >= 0 && lane == __ffs(peers) - 1) sh.hist[wid][l] += __popc(peers);
                __syncwarp();
            }
            csync<CS>();
            if (rank == 0) {
                // label totals over the cluster, their prefix, then every (rank, warp)
                // count replaced by its running offset (written into the owning block)
                for (int l = tid; l < k; l += kBT) {
                    int tot = 0;
                    for (int q2 = 0; q2 < CS; ++q2) {
                        const int(*hq)[kBMaxK] = CS > 1 ? cg::this_cluster().map_shared_rank(sh.hist, q2) : sh.hist;
                        for (int i = 0; i < kBW; ++i) tot += hq[i][l];
                    }
                    sh.wl_tot[l] = tot;
                }
                __syncthreads();
                if (tid == 0) {
                    int acc = 0;
                    for (int l = 0; l < k; ++l) {
                        sh.base[l] = acc;
                        acc += sh.wl_tot[l];
                    }
                    sh.base[k] = acc;
                }
                __syncthreads();
                for (int l = tid; l < k; l += kBT) {
                    int run2 = sh.base[l];
                    for (int q2 = 0; q2 < CS; ++q2) {
                        int(*hq)[kBMaxK] = CS > 1 ? cg::this_cluster().map_shared_rank(sh.hist, q2) : sh.hist;
                        for (int i = 0; i < kBW; ++i) {
                            const int c = hq[i][l];
                            hq[i][l] = run2;
                            run2 += c;
                        }
                    }
                }
                __syncthreads();
                if (CS > 1)
                    for (int q2 = 1; q2 < CS; ++q2) {
                        int *bq = cg::this_cluster().map_shared_rank(sh.base, q2);
                        for (int l = tid; l <= k; l += kBT) bq[l] = sh.base[l];
                    }
            }
            csync<CS>();
            for (int64_t c0 = w0; c0 < w1; c0 += 32) {
                const int64_t pt = c0 + lane;
                const int l = pt < w1 ? lab[pt] : -1;
                const unsigned peers = __match_any_sync(0xffffffffu, l);
                if (l >= 0) perm[sh.hist[wid][l] + __popc(peers & ((1u << lane) - 1u))] = (int32_t)pt;
                __syncwarp();
                if (l >= 0 && lane == __ffs(peers) - 1) sh.hist[wid][l] += __popc(peers);
                __syncwarp();
            }
            csync<CS>();
            // centroids: member coordinates in ascending point order, compensated FP32;
            // the (center, coordinate) pairs are shared out over the cluster
            for (int64_t pq = (int64_t)rank * kBT + tid; pq < (int64_t)k * d; pq += (int64_t)CS * kBT) {
                const int j = (int)(pq / d), qq = (int)(pq % d);
                const int b0 = sh.base[j], b1 = sh.base[j + 1];
                if (b1 == b0) continue;   // an empty cluster keeps its center
                float s = 0.f, c = 0.f;
                for (int i = b0; i < b1; ++i) two_sum_add(s, c, X[(int64_t)perm[i] * d + qq]);
                C[pq] = (float)(((double)s + (double)c) / (double)(b1 - b0));
            }
            csync<CS>();
        }
        res.iters = it;
        res.final_cost = cost;
        if (a.labels_out)
            for (int64_t pt = r0 + tid; pt < r1; pt += kBT) a.labels_out[P.l_off + pt] = lab[pt];
    }
    if (a.cand_out)
        for (int j = rank * kBT + tid; j < m && j < P.cap_total; j += CS * kBT) a.cand_out[P.cand_off + j] = cand[j];
    if (a.w_out && status != KMPAR_ERR_CAPACITY)
        for (int j = rank * kBT + tid; j < m; j += CS * kBT) a.w_out[P.cand_off + j] = w[j];
    const unsigned long long nr = csum<CS>(sh.s_near, &sh.s_uslot);
    const unsigned long long nf = csum<CS>(sh.s_fp64, &sh.s_uslot);
    const unsigned long long nrc = csum<CS>(sh.s_rnear, &sh.s_uslot);
    if (rank == 0 && tid == 0) {
        res.status = status;
        res.sample_near = nr;
        res.argmin_fp64 = nf;
        res.recluster_near = nrc;
        a.res[pi] = res;
    }
}

}  // namespace
}  // namespace kmp

// ------------------------------------------------------------------ host side
namespace kmp {
namespace {

// l + 10 sqrt(l) + 64 (the round count is a sum of independent draws with mean at
// most l and variance at most l), lowered by KMPAR_ROUND_CAPACITY when set
int batch_round_capacity(double ell) {
    double c = ell + 10.0 * std::sqrt(ell) + 64.0;
    if (c > 2.0e9) c = 2.0e9;
    int cap = (int)std::ceil(c);
    if (const char *v = std::getenv("KMPAR_ROUND_CAPACITY")) {
        char *end = nullptr;
        const unsigned long long x = std::strtoull(v, &end, 10);
        if (*v && end && *end == 0 && x > 0 && x < (unsigned long long)cap) cap = (int)x;
    }
    return cap;
}

kmpar_status batch_fail(kmpar_status s, const std::string &m) {
    kmp::set_thread_error(m);
    return s;
}

// rows per block a problem is cut into: problems larger than this run as a cluster
// (kmpar_batch_set_split; 0: never split)
std::atomic<int64_t> g_rows_per_block{25000};

int cluster_size(int64_t n) {
    const int64_t rpb = g_rows_per_block.load(std::memory_order_relaxed);
    int cs = 1;
    while (rpb > 0 && cs < 8 && (n + cs - 1) / cs > rpb) cs *= 2;
    return cs;
}

template <int DP, int CS>
cudaError_t launch_cs(const kmp::BArgs &a, int first, int count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    if (CS == 1) {
        kmp::batch_kernel<DP, 1><<<count, kmp::kBT, 0, s>>>(a, first);
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(count * CS));
        cfg.blockDim = dim3(kmp::kBT);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, kmp::batch_kernel<DP, CS>, a, first);
        if (e != cudaSuccess) return e;
    }
    kmp::count_launches(1);
    return cudaGetLastError();
}

template <int DP>
cudaError_t launch_class(const kmp::BArgs &a, int cs, int first, int count, cudaStream_t s) {
    switch (cs) {
        case 1: return launch_cs<DP, 1>(a, first, count, s);
        case 2: return launch_cs<DP, 2>(a, first, count, s);
        case 4: return launch_cs<DP, 4>(a, first, count, s);
        case 8: return launch_cs<DP, 8>(a, first, count, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace kmp

extern "C" {

kmpar_status kmpar_batch_set_split(int32_t rows_per_block) {
    if (rows_per_block < 0) return kmp::batch_fail(KMPAR_ERR_ARG, "rows_per_block < 0");
    kmp::g_rows_per_block.store(rows_per_block, std::memory_order_relaxed);
    return KMPAR_OK;
}

int64_t kmpar_batch_cand_capacity(double ell, int32_t rounds) {
    if (!(ell > 0.0) || rounds < 0) return 0;
    return 1 + (int64_t)rounds * kmp::batch_round_capacity(ell);
}

kmpar_status kmpar_batch_run(const float *X, const kmpar_problem *problems, int32_t count, float *centers_out,
                             int32_t *labels_out, int32_t *cand_out, int64_t *w_out, kmpar_problem_result *results,
                             void *stream) {
    using namespace kmp;
    if (count < 0 || (count > 0 && (!X || !problems || !centers_out || !results)))
        return batch_fail(KMPAR_ERR_ARG, "NULL pointer or negative count");
    if (count == 0) return KMPAR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<BProb> hp((size_t)count);
    std::vector<double> work((size_t)count);
    int64_t p_tot = 0, m_tot = 0;
    for (int i = 0; i < count; ++i) {
        const kmpar_problem &q = problems[i];
        if (q.n < 1 || q.n >= (int64_t)INT32_MAX || q.d < 1 || q.d > 128 || q.k < 1 || q.k > kBMaxK ||
            !(q.ell > 0.0) || !std::isfinite(q.ell) || q.rounds < 0 || q.rounds > kBMaxRounds || q.max_iter < 0 ||
            q.x_offset < 0 || q.c_offset < 0 || q.l_offset < 0 || q.cand_offset < 0)
            return batch_fail(KMPAR_ERR_ARG, "problem " + std::to_string(i) + ": argument out of range");
        const int cap = batch_round_capacity(q.ell);
        if (cap > kBMaxCap)
            return batch_fail(KMPAR_ERR_UNSUPPORTED,
                              "problem " + std::to_string(i) + ": l + 10 sqrt(l) + 64 exceeds 4096 per round");
        BProb &b = hp[(size_t)i];
        b.x_off = q.x_offset; b.n = q.n; b.d = q.d; b.k = q.k; b.ell = q.ell; b.rounds = q.rounds;
        b.max_iter = q.max_iter; b.seed = q.seed; b.c_off = q.c_offset; b.l_off = q.l_offset;
        b.cand_off = q.cand_offset;
        b.cap_round = cap;
        b.cap_total = 1 + q.rounds * cap;
        b.p_off = p_tot;
        b.m_off = m_tot;
        p_tot += q.n;
        m_tot += b.cap_total;
        // distance evaluations of the rounds and of Lloyd, times the padded dimension
        const int dp = q.d <= 32 ? 32 : (q.d <= 64 ? 64 : 128);
        work[(size_t)i] = (double)q.n * dp * (1.0 + q.rounds * q.ell + (double)(q.max_iter + 1) * q.k);
    }
    // one launch per (dimension class, cluster size), largest problems first in each
    std::vector<int32_t> order;
    order.reserve((size_t)count);
    struct Cls { int dp, cs, first, count; };
    std::vector<Cls> classes;
    for (int c = 0; c < 3; ++c) {
        const int lo = c == 0 ? 1 : (c == 1 ? 33 : 65), hi = c == 0 ? 32 : (c == 1 ? 64 : 128);
        for (int cs = 8; cs >= 1; cs /= 2) {
            std::vector<int32_t> ids;
            for (int i = 0; i < count; ++i)
                if (problems[i].d >= lo && problems[i].d <= hi && cluster_size(problems[i].n) == cs) ids.push_back(i);
            if (ids.empty()) continue;
            std::stable_sort(ids.begin(), ids.end(), [&](int32_t x, int32_t y) { return work[x] > work[y]; });
            classes.push_back({c == 0 ? 32 : (c == 1 ? 64 : 128), cs, (int)order.size(), (int)ids.size()});
            order.insert(order.end(), ids.begin(), ids.end());
        }
    }
    // one device block holds the table, the order, the results and the work space
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t o_probs = 0;
    const size_t o_order = o_probs + up(sizeof(BProb) * (size_t)count);
    const size_t o_res = o_order + up(sizeof(int32_t) * (size_t)count);
    const size_t o_d2 = o_res + up(sizeof(BRes) * (size_t)count);
    const size_t o_idx = o_d2 + up(sizeof(float) * (size_t)p_tot);
    const size_t o_lab = o_idx + up(sizeof(int32_t) * (size_t)p_tot);
    const size_t o_perm = o_lab + up(sizeof(int32_t) * (size_t)p_tot);
    const size_t o_cand = o_perm + up(sizeof(int32_t) * (size_t)p_tot);
    const size_t o_w = o_cand + up(sizeof(int32_t) * (size_t)m_tot);
    const size_t o_rd2 = o_w + up(sizeof(int32_t) * (size_t)m_tot);
    const size_t total = o_rd2 + up(sizeof(float) * (size_t)m_tot);
    unsigned char *ws = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&ws), total, s);
    if (e != cudaSuccess)
        return batch_fail(e == cudaErrorMemoryAllocation ? KMPAR_ERR_OOM : KMPAR_ERR_CUDA,
                          std::string("batch work space: ") + cudaGetErrorString(e));
    std::vector<BRes> hres((size_t)count);
    const int nside = (int)classes.size() - 1;
    std::vector<cudaStream_t> side((size_t)std::max(0, nside), nullptr);
    std::vector<cudaEvent_t> ev_join((size_t)std::max(0, nside), nullptr);
    cudaEvent_t ev_fork = nullptr;
    BArgs a{};
    a.X = X;
    a.probs = reinterpret_cast<const BProb *>(ws + o_probs);
    a.order = reinterpret_cast<const int32_t *>(ws + o_order);
    a.centers = centers_out;
    a.labels_out = labels_out;
    a.cand_out = cand_out;
    a.w_out = reinterpret_cast<long long *>(w_out);
    a.res = reinterpret_cast<BRes *>(ws + o_res);
    a.D2 = reinterpret_cast<float *>(ws + o_d2);
    a.idx = reinterpret_cast<int32_t *>(ws + o_idx);
    a.lab = reinterpret_cast<int32_t *>(ws + o_lab);
    a.perm = reinterpret_cast<int32_t *>(ws + o_perm);
    a.cand = reinterpret_cast<int32_t *>(ws + o_cand);
    a.w = reinterpret_cast<int32_t *>(ws + o_w);
    a.rD2 = reinterpret_cast<float *>(ws + o_rd2);
    e = cudaMemcpyAsync(ws + o_probs, hp.data(), sizeof(BProb) * (size_t)count, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws + o_order, order.data(), sizeof(int32_t) * (size_t)count, cudaMemcpyHostToDevice, s);
    // the classes run concurrently: the caller's stream and side streams forked from
    // it and joined back (also valid inside a stream capture)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
    for (int i = 0; i < nside && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&side[(size_t)i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_join[(size_t)i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev_fork, s);
    for (int i = 0; i < nside && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(side[(size_t)i], ev_fork, 0);
    for (size_t c = 0; c < classes.size() && e == cudaSuccess; ++c) {
        const Cls &q = classes[c];
        cudaStream_t cs = c == 0 ? s : side[c - 1];
        if (q.dp == 32) e = launch_class<32>(a, q.cs, q.first, q.count, cs);
        else if (q.dp == 64) e = launch_class<64>(a, q.cs, q.first, q.count, cs);
        else e = launch_class<128>(a, q.cs, q.first, q.count, cs);
    }
    for (int i = 0; i < nside && e == cudaSuccess; ++i) {
        e = cudaEventRecord(ev_join[(size_t)i], side[(size_t)i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_join[(size_t)i], 0);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hres.data(), ws + o_res, sizeof(BRes) * (size_t)count, cudaMemcpyDeviceToHost, s);
    const cudaError_t ef = cudaFreeAsync(ws, s);
    if (e == cudaSuccess) e = ef;
    const cudaError_t es = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = es;
    for (int i = 0; i < nside; ++i) {
        if (side[(size_t)i]) cudaStreamDestroy(side[(size_t)i]);
        if (ev_join[(size_t)i]) cudaEventDestroy(ev_join[(size_t)i]);
    }
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (e != cudaSuccess) return batch_fail(KMPAR_ERR_CUDA, std::string("batch kernels: ") + cudaGetErrorString(e));
    kmpar_status worst = KMPAR_OK;
    for (int i = 0; i < count; ++i) {
        const BRes &r = hres[(size_t)i];
        kmpar_problem_result &o = results[i];
        o.m = r.m;
        o.seed_cost = r.seed_cost;
        o.final_cost = r.final_cost;
        o.iters = r.iters;
        o.status = r.status;
        o.sample_near = (int64_t)r.sample_near;
        o.argmin_fp64 = (int64_t)r.argmin_fp64;
        o.recluster_near = (int64_t)r.recluster_near;
        if (r.status == KMPAR_ERR_CAPACITY) worst = KMPAR_ERR_CAPACITY;
        else if (r.status == KMPAR_WARN_FEW_CANDIDATES && worst == KMPAR_OK) worst = KMPAR_WARN_FEW_CANDIDATES;
    }
    if (worst == KMPAR_ERR_CAPACITY) kmp::set_thread_error("a problem's round drew more points than its capacity");
    return worst;
}

}  // extern "C"
