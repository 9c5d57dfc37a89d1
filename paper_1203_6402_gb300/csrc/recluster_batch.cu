// recluster_batch.cu -- Alg. 2 step 8 (weighted k-means++: Alg. 1 with
// multiplicities, Sec. 4.2), the draws after the first taken in batches by
// rejection from a stale snapshot of D^2.
//
// The law is the one of the one-draw-at-a-time kernels: every draw picks j with
// probability w_j D^2(j) / sum_j w_j D^2(j), D^2 to all centers drawn before it.
// A snapshot S = D^2 fixes the masses w_j S_j; 2B proposals are drawn from them
// (inverse CDF); in proposal order, proposal j is kept iff v S_j < D(j), D(j) the
// smaller of S_j and the distances from j to the centers kept since the snapshot.
// A proposal is made with probability w_j S_j / sum and kept with probability
// D(j) / S_j, so a kept j has probability proportional to w_j D(j).  A snapshot
// keeps up to B draws, so k draws take about k / B snapshots instead of k
// dependent steps.
//
// Per snapshot, five launches on the context's stream and no wait between CTAs:
//   rs_update_kernel   D^2 of every candidate against the centers kept in the last
//                      snapshot (a sum stops once it reaches D^2: sums of
//                      non-negative terms never decrease), masses w D^2 as double
//                      floats, the total of each chunk of 32 candidates;
//   rs_scan_kernel     one block: the chunk totals' inclusive prefix sums (ascending);
//   rs_propose_kernel  one warp per proposal i: u from counter (p + i, 0, 0, 5),
//                      target u * total, then the chunk from the prefix sums and the
//                      candidate from the chunk's masses;
//   rs_pair_kernel     squared distances between the proposals (each pair once);
//   rs_accept_kernel   one warp walks the proposals in order, v from counter
//                      (p + i, 1, 0, 5), and appends the kept ones to the chosen list.
// Draw 0 is the one-at-a-time kernels' draw 0 (mass w, counter (0, 0, 0, 3)).
// Random numbers, prefix order and near-tie flags follow the FP64 definition; the
// device sums are FP32 distances and double-float masses, so a decision can differ
// from exact arithmetic only where a near-tie flag is raised.
#include <algorithm>

#include "dfloat.cuh"
#include "kmpar_internal.cuh"

namespace kmp {

namespace {

constexpr uint32_t TAG_RECLUSTER_RS = 5u;
constexpr int kUpdWarps = 8;                       // update block: 32 candidates x 8 groups of 8 centers
constexpr int kPropWarps = 4;                      // proposals per propose block
constexpr int kScanThreads = 1024;                 // the chunk-prefix block
constexpr int kAcceptThreads = 256;

struct RsCtl {
    int t;                   // centers chosen so far
    int first_new;           // chosen[first_new .. t): kept in the last snapshot, not yet in D^2
    int done;                // t == k, or the mass ran out
    int init;                // 1: the next update sets D^2 from chosen[0]
    int zero;                // the snapshot's total mass was 0
    int pending;             // a near event since the last kept draw
    unsigned long long p;    // counter of the snapshot's first proposal
};


struct RsProp {
    int j;        // proposed candidate
    int near;     // its target within 1e-6 total of a prefix boundary (or a fallback)
    float S;      // its snapshot D^2
    float pad;
    double v;     // acceptance uniform
};

// partial distances of candidate j (coordinates from the transposed copy: one
// coalesced load per coordinate for a warp's 32 candidates) to the nr <= 8 centers
// whose rows are C[rows[g]] (the same address in every lane: broadcast loads that
// stay in L1), coordinates in ascending order, each sum t = y - c, s = fma(t, t, s).
// Stops once every sum has reached lim (it can then no longer lower the minimum:
// sums of non-negative terms never decrease); s[g] = +inf for g >= nr.
template <bool VEC>
__device__ __forceinline__ void dist2_8(const float *__restrict__ CT, int mp, int j, const float *__restrict__ C,
                                        const int32_t *rows, int nr, int d, float lim, float (&s)[8]) {
    const float *c[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        s[g] = g < nr ? 0.f : __int_as_float(0x7f800000);
        c[g] = C + (size_t)(g < nr ? rows[g] : rows[0]) * d;
    }
    int q = 0;
    for (; q + 16 <= d; q += 16) {
        float y[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) y[u] = __ldg(CT + (size_t)(q + u) * mp + j);
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            if (g < nr) {
                if (VEC) {
#pragma unroll
                    for (int u = 0; u < 16; u += 4) {
                        const float4 c4 = __ldg(reinterpret_cast<const float4 *>(c[g] + q + u));
                        float t = __fsub_rn(y[u], c4.x);
                        s[g] = __fmaf_rn(t, t, s[g]);
                        t = __fsub_rn(y[u + 1], c4.y);
                        s[g] = __fmaf_rn(t, t, s[g]);
                        t = __fsub_rn(y[u + 2], c4.z);
                        s[g] = __fmaf_rn(t, t, s[g]);
                        t = __fsub_rn(y[u + 3], c4.w);
                        s[g] = __fmaf_rn(t, t, s[g]);
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const float t = __fsub_rn(y[u], __ldg(c[g] + q + u));
                        s[g] = __fmaf_rn(t, t, s[g]);
                    }
                }
            }
        }
        bool done = true;
#pragma unroll
        for (int g = 0; g < 8; ++g) done &= !(s[g] < lim);
        if (done) return;
    }
    for (; q < d; ++q) {
        const float y = __ldg(CT + (size_t)q * mp + j);
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            if (g < nr) {
                const float t = __fsub_rn(y, __ldg(c[g] + q));
                s[g] = __fmaf_rn(t, t, s[g]);
            }
        }
    }
}

// ||a - b||^2 between two candidate rows, stopping once the sum reaches lim
__device__ __forceinline__ float dist2_rows_lim(const float *__restrict__ a, const float *__restrict__ b, int d,
                                                float lim) {
    float s = 0.f;
    int q = 0;
    for (; q + 16 <= d; q += 16) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const float t = __fsub_rn(__ldg(a + q + u), __ldg(b + q + u));
            s = __fmaf_rn(t, t, s);
        }
        if (s >= lim) return s;
    }
    for (; q < d; ++q) {
        const float t = __fsub_rn(__ldg(a + q), __ldg(b + q));
        s = __fmaf_rn(t, t, s);
    }
    return s;
}

// One block per chunk of 32 candidates: D^2 against the centers kept in the last
// snapshot, warp w taking centers 8w .. 8w+7 of them (the 8 warps read the same
// candidate coordinates, which L1 then serves), the minimum over the warps, and the
// chunk's mass total gch (FP64 of the double-float warp scan).  FIRST: no D^2, mass
// w.  Up to 64 new centers (8 warps x 8).
template <bool FIRST, bool VEC>
__global__ void __launch_bounds__(kUpdWarps * 32) rs_update_kernel(const float *__restrict__ C,
                                                                     const float *__restrict__ CT, int mp,
                                                                     const long long *__restrict__ w,
                                                                     const DevState *st, int d,
                                                                     const int32_t *__restrict__ chosen,
                                                                     const RsCtl *ctl, float *__restrict__ D2,
                                                                     float2 *__restrict__ gch) {
    __shared__ float s_min[kUpdWarps][32];
    if (ctl->done) return;
    const int m = st->m;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + lane;
    float dj = __int_as_float(0x7f800000);
    if (!FIRST) {
        const bool init = ctl->init != 0;
        const int a0 = init ? 0 : ctl->first_new, a1 = init ? 1 : ctl->t;
        if (j < m && !init) dj = D2[j];
        float best = __int_as_float(0x7f800000);
        const int c0 = a0 + 8 * wid;
        if (c0 < a1 && j < m) {
            float s8[8];
            dist2_8<VEC>(CT, mp, j, C, chosen + c0, min(8, a1 - c0), d, dj, s8);
#pragma unroll
            for (int g = 0; g < 8; ++g) best = fminf(best, s8[g]);
        }
        s_min[wid][lane] = best;
        __syncthreads();
    }
    if (wid != 0) return;
    Df e = {0.f, 0.f};
    if (j < m) {
        const float2 wv = weight_split(w[j]);
        if (FIRST) {
            e = df_mass(wv, 0.f, true);
        } else {
#pragma unroll
            for (int w2 = 0; w2 < kUpdWarps; ++w2) dj = fminf(dj, s_min[w2][lane]);
            D2[j] = dj;
            e = df_mass(wv, dj, false);
        }
    }
    const Df incl = warp_incl_scan_df(e, lane);
    if (lane == 31) gch[blockIdx.x] = make_float2(incl.hi, incl.lo);
}

// One block: inclusive prefix sums of the chunk totals in ascending order (each
// thread a contiguous range, warp scans, then a scan of the warp totals), double
// floats on the FP32 pipes; the same values serve every proposal of the snapshot;
// gincl[nchunk] = the total.
__global__ void __launch_bounds__(kScanThreads) rs_scan_kernel(const RsCtl *ctl, const float2 *__restrict__ gch,
                                                              int nchunk, float2 *__restrict__ gincl) {
    __shared__ float2 s_w[kScanThreads / 32];
    if (ctl->done) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int per = (nchunk + kScanThreads - 1) / kScanThreads;
    const int c0 = min(nchunk, (int)threadIdx.x * per), c1 = min(nchunk, c0 + per);
    // (16 loads in flight per thread; adding a zero double float is exact)
    Df ls = {0.f, 0.f};
    for (int b = c0; b < c1; b += 16) {
        float2 g[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) g[r] = b + r < c1 ? gch[b + r] : make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < 16; ++r) ls = df_add(ls, Df{g[r].x, g[r].y});
    }
    const Df wi = warp_incl_scan_df(ls, lane);
    if (lane == 31) s_w[wid] = make_float2(wi.hi, wi.lo);
    __syncthreads();
    if (wid == 0) {
        // exclusive prefix of the warp totals
        const Df v = lane < kScanThreads / 32 ? Df{s_w[lane].x, s_w[lane].y} : Df{0.f, 0.f};
        const Df vi = warp_incl_scan_df(v, lane);
        Df vx = {__shfl_up_sync(0xffffffffu, vi.hi, 1), __shfl_up_sync(0xffffffffu, vi.lo, 1)};
        if (lane == 0) vx = Df{0.f, 0.f};
        __syncwarp();
        if (lane < kScanThreads / 32) s_w[lane] = make_float2(vx.hi, vx.lo);
    }
    __syncthreads();
    // exclusive prefix of this thread's range
    Df ex = {__shfl_up_sync(0xffffffffu, wi.hi, 1), __shfl_up_sync(0xffffffffu, wi.lo, 1)};
    if (lane == 0) ex = Df{0.f, 0.f};
    Df run = df_add(Df{s_w[wid].x, s_w[wid].y}, ex);
    for (int b = c0; b < c1; b += 16) {
        float2 g[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) g[r] = b + r < c1 ? gch[b + r] : make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            if (b + r < c1) {
                run = df_add(run, Df{g[r].x, g[r].y});
                gincl[b + r] = make_float2(run.hi, run.lo);
            }
        }
    }
    if (threadIdx.x == kScanThreads - 1) gincl[nchunk] = make_float2(run.hi, run.lo);
}

// one warp per proposal: the candidate whose prefix interval holds u * total
template <bool FIRST>
__global__ void __launch_bounds__(32 * kPropWarps) rs_propose_kernel(const long long *__restrict__ w,
                                                                    const float *__restrict__ D2,
                                                                    const DevState *st,
                                                                    const float2 *__restrict__ gch,
                                                                    const float2 *__restrict__ gincl, int nchunk,
                                                                    RsCtl *ctl, uint64_t seed, int P,
                                                                    RsProp *__restrict__ props) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kPropWarps + (threadIdx.x >> 5);
    if (i >= P || ctl->done) return;
    const int m = st->m;
    auto dv = [](float2 v) { return (double)v.x + (double)v.y; };
    const double total = dv(gincl[nchunk]);
    if (!(total > 0.0)) {
        if (i == 0 && lane == 0) ctl->zero = 1;
        return;
    }
    const uint64_t ctr = FIRST ? 0ull : ctl->p + (uint64_t)i;
    const double u = uniform53(ctr, 0, FIRST ? TAG_RECLUSTER : TAG_RECLUSTER_RS, seed);
    const double target = __dmul_rn(u, total);
    int near = 0;
    // chunk: the first with positive mass whose inclusive prefix exceeds the target,
    // found among 32 segment ends and then within the segment; if rounding leaves
    // none, the last chunk with positive mass (a chunk with positive mass holds a
    // candidate with positive mass, so the pick below is always a real candidate)
    int ch = -1;
    {
        const int seg = (nchunk + 31) / 32;
        const int e = min(nchunk, (lane + 1) * seg) - 1;
        const bool have = lane * seg < nchunk;
        const unsigned hit = __ballot_sync(0xffffffffu, have && dv(gincl[e]) > target);
        if (hit) {
            const int L = __ffs(hit) - 1;
            const int b0 = L * seg, b1 = min(nchunk, b0 + seg);
            for (int b = b0; b < b1 && ch < 0; b += 32) {
                const int c = b + lane;
                const unsigned h2 = __ballot_sync(0xffffffffu, c < b1 && dv(gincl[c]) > target && gch[c].x > 0.f);
                if (h2) ch = b + __ffs(h2) - 1;
            }
        }
        if (ch < 0) {
            // the last chunk whose total is positive
            for (int b = (nchunk - 1) & ~31; b >= 0 && ch < 0; b -= 32) {
                const int c = b + lane;
                const unsigned h2 = __ballot_sync(0xffffffffu, c < nchunk && gch[c].x > 0.f);
                if (h2) ch = b + 31 - __clz(h2);
            }
            near = 1;
        }
    }
    const double pre_c = ch > 0 ? dv(gincl[ch - 1]) : 0.0;
    // candidate within the chunk: the same masses as the update kernel's
    const int j = ch * 32 + lane;
    Df e = {0.f, 0.f};
    if (j < m) e = df_mass(weight_split(w[j]), FIRST ? 0.f : D2[j], FIRST);
    const Df inclf = warp_incl_scan_df(e, lane);
    const double ev = df_to_double(e), ic = df_to_double(inclf);
    const double cum = __dadd_rn(pre_c, ic), cum0 = __dadd_rn(pre_c, __dsub_rn(ic, ev));
    // (a candidate without mass is never the first to pass the target)
    const unsigned hit = __ballot_sync(0xffffffffu, j < m && ev > 0.0 && cum > target);
    int pick;
    if (hit) {
        const int hl = __ffs(hit) - 1;
        pick = ch * 32 + hl;
        const int nr = fabs(target - cum0) <= 1e-6 * total || fabs(cum - target) <= 1e-6 * total;
        near |= __shfl_sync(0xffffffffu, nr, hl);
    } else {
        const unsigned pos = __ballot_sync(0xffffffffu, j < m && ev > 0.0);
        pick = ch * 32 + (pos ? 31 - __clz(pos) : 0);
        near = 1;
    }
    if (lane == 0) {
        RsProp pr;
        pr.j = pick;
        pr.near = near;
        pr.S = FIRST ? 0.f : D2[pick];
        pr.pad = 0.f;
        pr.v = FIRST ? 0.0 : uniform53(ctl->p + (uint64_t)i, 1, TAG_RECLUSTER_RS, seed);
        props[i] = pr;
    }
}

// Dpp[i' P + i] = ||c_{j_i} - c_{j_i'}||^2 for i' < i, stopping at S_i (row i' holds
// the distances from proposal i' to the later proposals, read in a row when i' is kept)
__global__ void __launch_bounds__(128) rs_pair_kernel(const float *__restrict__ C, int d, const RsProp *props,
                                                      int P, const RsCtl *ctl, float *__restrict__ Dpp) {
    if (ctl->done || ctl->zero) return;
    const int i = blockIdx.x;
    const RsProp pi = props[i];
    const float *a = C + (size_t)pi.j * d;
    for (int i2 = threadIdx.x; i2 < i; i2 += blockDim.x)
        Dpp[(size_t)i2 * P + i] = dist2_rows_lim(a, C + (size_t)props[i2].j * d, d, pi.S);
}

// the proposals in order: kept iff v S_j < D(j); FIRST: proposal 0 is draw 0.
// The test v S_j < D(j) (FP64 product, FP32 D) is the FP32 test D(j) >= T_j with
// T_j the smallest float above v S_j, and the near window |v S_j - D(j)| <=
// 1e-4 S_j is [lo_j, hi_j] rounded outwards to floats: both are set up for all
// proposals at once, and one warp then jumps from one kept proposal to the next
// (a ballot over the proposals after the last kept one finds the first that passes;
// the ones before it fail whatever is kept later, since D only decreases).
template <bool FIRST>
__global__ void __launch_bounds__(kAcceptThreads) rs_accept_kernel(const RsProp *props, int P, int B,
                                                                  const float *__restrict__ Dpp, RsCtl *ctl,
                                                                  int32_t *__restrict__ chosen, DevState *st,
                                                                  int k) {
    // the P x P pair distances (row i': proposal i' to the later ones), then per
    // proposal D(j), T_j, lo_j, hi_j, j and its target's near flag
    extern __shared__ __align__(16) float dsm[];
    __shared__ int s_zero;
    if (ctl->done) return;
    if (threadIdx.x == 0) s_zero = ctl->zero;
    __syncthreads();
    if (s_zero) {
        // the positive mass ran out: the remaining draws repeat chosen[0]
        const int t = ctl->t;
        for (int a = t + threadIdx.x; a < k; a += blockDim.x) chosen[a] = t > 0 ? chosen[0] : 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            st->warn = 1;
            ctl->t = k;
            ctl->done = 1;
        }
        return;
    }
    if (FIRST) {
        if (threadIdx.x == 0) {
            const RsProp p0 = props[0];
            chosen[0] = p0.j;
            if (p0.near) atomicAdd(&st->recluster_near, 1ull);
            ctl->t = 1;
            ctl->first_new = 0;
            ctl->init = 1;
            ctl->p = 0;
            if (k <= 1) ctl->done = 1;
        }
        return;
    }
    float *dpp = dsm;
    float *dcur = dpp + (size_t)P * P;
    float *thr = dcur + P;
    float *nlo = thr + P;
    float *nhi = nlo + P;
    int *sj = reinterpret_cast<int *>(nhi + P);
    int *snr = sj + P;
    {
        // the whole P x P block (P is even: rows of float4; row i' is read from i' + 1 on)
        const float4 *src = reinterpret_cast<const float4 *>(Dpp);
        float4 *dst = reinterpret_cast<float4 *>(dpp);
        const int n4 = P * P / 4;
        // 16 loads in flight per thread before their stores
        for (int f0 = 0; f0 < n4; f0 += 16 * kAcceptThreads) {
            float4 v[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const int f = f0 + r * kAcceptThreads + threadIdx.x;
                if (f < n4) v[r] = __ldcg(src + f);
            }
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const int f = f0 + r * kAcceptThreads + threadIdx.x;
                if (f < n4) dst[f] = v[r];
            }
        }
    }
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const RsProp pr = props[i];
        const double S = (double)pr.S;
        const double lhs = __dmul_rn(pr.v, S);
        float T = __double2float_ru(lhs);
        if ((double)T == lhs) T = __int_as_float(__float_as_int(T) + 1);   // lhs > 0: the next float up
        const double win = __dmul_rn(1e-4, S);
        dcur[i] = pr.S;
        thr[i] = T;
        nlo[i] = __double2float_rd(__dsub_rn(lhs, win));
        nhi[i] = __double2float_ru(__dadd_rn(lhs, win));
        sj[i] = pr.j;
        snr[i] = pr.near;
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    // lane l holds proposals l, l + 32, l + 64, l + 96 in registers
    constexpr int R = kRsMaxProposals / 32;
    const int lane = threadIdx.x;
    float rd[R], rt[R], rlo[R], rhi[R];
    bool rnr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = r * 32 + lane;
        const bool ok = i < P;
        rd[r] = ok ? dcur[i] : 0.f;
        rt[r] = ok ? thr[i] : __int_as_float(0x7f800000);
        rlo[r] = ok ? nlo[i] : 1.f;
        rhi[r] = ok ? nhi[i] : 0.f;
        rnr[r] = ok && snr[i] != 0;
    }
    const int t0 = ctl->t;
    int t = t0, pending = ctl->pending, nnear = 0, cur = 0;
    while (t < k && t - t0 < B && cur < P) {
        // the first proposal at or after cur that passes (dcur >= T), and the near
        // flags of the proposals examined up to it
        int first = P;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = r * 32 + lane;
            const unsigned b = __ballot_sync(0xffffffffu, i >= cur && i < P && rd[r] >= rt[r]);
            if (b && first == P) first = r * 32 + __ffs(b) - 1;
        }
        const int last = first < P ? first : P - 1;
        bool nr = false;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = r * 32 + lane;
            if (i >= cur && i <= last) nr |= rnr[r] || (rd[r] >= rlo[r] && rd[r] <= rhi[r]);
        }
        if (__any_sync(0xffffffffu, nr)) pending = 1;
        if (first == P) break;   // none passes: every remaining proposal was examined
        if (lane == 0) chosen[t] = sj[first];
        nnear += pending;
        pending = 0;
        ++t;
        // D of the later proposals: the kept one's row of pair distances
        const float *row = dpp + (size_t)first * P;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = r * 32 + lane;
            if (i > first && i < P) rd[r] = fminf(rd[r], row[i]);
        }
        cur = first + 1;
    }
    if (lane == 0) {
        ctl->first_new = t0;
        ctl->init = 0;
        ctl->t = t;
        ctl->pending = pending;
        ctl->p += (unsigned long long)P;
        if (t >= k) ctl->done = 1;
        if (nnear) atomicAdd(&st->recluster_near, (unsigned long long)nnear);
        atomicAdd(&st->recluster_snapshots, 1ull);
    }
}

__global__ void rs_gather_kernel(const float *__restrict__ C, int d, const int32_t *__restrict__ chosen, int k,
                                 float *__restrict__ centers) {
    const size_t total = (size_t)k * d;
    for (size_t f = (size_t)blockIdx.x * blockDim.x + threadIdx.x; f < total; f += (size_t)gridDim.x * blockDim.x) {
        const size_t a = f / d, q = f - a * d;
        centers[f] = C[(size_t)chosen[a] * d + q];
    }
}

}  // namespace

size_t recluster_batch_bytes() {
    return 256 + sizeof(RsProp) * kRsMaxProposals + sizeof(float) * (size_t)kRsMaxProposals * kRsMaxProposals;
}

cudaError_t launch_recluster_batch(Ctx &c, float *centers) {
    cudaError_t e;
    const int B = c.rs_batch, P = 2 * B;
    if (B < 1 || P > kRsMaxProposals || !c.rCT || !c.rs_buf) return cudaErrorInvalidValue;
    const int mp = (c.cap_total + 31) / 32 * 32;
    const int nchunk = (c.cap_total + 31) / 32;   // one update block per chunk of 32 candidates
    static_assert(kRsMaxBatch <= 8 * kUpdWarps, "update block: 8 warps x 8 new centers");
    if ((e = launch_transpose_cand(c)) != cudaSuccess) return e;
    RsCtl *ctl = reinterpret_cast<RsCtl *>(c.rs_buf);
    RsProp *props = reinterpret_cast<RsProp *>(reinterpret_cast<char *>(c.rs_buf) + 256);
    float *Dpp = reinterpret_cast<float *>(props + kRsMaxProposals);
    // chunk totals and their inclusive prefix sums (then the total), double floats,
    // in the chunk-mass buffer (2 nchunk + 2048 doubles)
    float2 *gch = reinterpret_cast<float2 *>(c.rc_cmass);
    float2 *gincl = gch + nchunk;
    const size_t acc_smem = sizeof(float) * ((size_t)P * P + 4 * P) + sizeof(int) * 2 * P;
    auto upd = c.d % 4 == 0 ? rs_update_kernel<false, true> : rs_update_kernel<false, false>;
    if (acc_smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(rs_accept_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)acc_smem)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(ctl, 0, sizeof(RsCtl), c.stream)) != cudaSuccess) return e;
    const int pgrid = (P + kPropWarps - 1) / kPropWarps;
    // draw 0
    rs_update_kernel<true, false><<<nchunk, 32 * kUpdWarps, 0, c.stream>>>(c.C, c.rCT, mp, c.w, c.st, c.d,
                                                                           c.chosen, ctl, c.rD2, gch);
    rs_scan_kernel<<<1, kScanThreads, 0, c.stream>>>(ctl, gch, nchunk, gincl);
    rs_propose_kernel<true><<<1, 32 * kPropWarps, 0, c.stream>>>(c.w, c.rD2, c.st, gch, gincl, nchunk, ctl, c.seed,
                                                                 1, props);
    rs_accept_kernel<true><<<1, kAcceptThreads, 0, c.stream>>>(props, 1, 1, Dpp, ctl, c.chosen, c.st, c.k);
    count_launches(4);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // snapshots: at least ceil((k - 1) / B); more while the proposals of a
    // snapshot keep fewer than B (each snapshot keeps at least its first proposal)
    int need = (c.k - 1 + B - 1) / B, launched = 0;
    while (need > 0) {
        for (int s = 0; s < need; ++s) {
            upd<<<nchunk, 32 * kUpdWarps, 0, c.stream>>>(c.C, c.rCT, mp, c.w, c.st, c.d, c.chosen, ctl, c.rD2, gch);
            rs_scan_kernel<<<1, kScanThreads, 0, c.stream>>>(ctl, gch, nchunk, gincl);
            rs_propose_kernel<false><<<pgrid, 32 * kPropWarps, 0, c.stream>>>(c.w, c.rD2, c.st, gch, gincl, nchunk,
                                                                              ctl, c.seed, P, props);
            rs_pair_kernel<<<P, 128, 0, c.stream>>>(c.C, c.d, props, P, ctl, Dpp);
            rs_accept_kernel<false><<<1, kAcceptThreads, acc_smem, c.stream>>>(props, P, B, Dpp, ctl, c.chosen,
                                                                               c.st, c.k);
        }
        count_launches(5 * need);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        launched += need;
        int h[4] = {0, 0, 0, 0};
        if ((e = cudaMemcpyAsync(h, ctl, sizeof(h), cudaMemcpyDeviceToHost, c.stream)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(c.stream)) != cudaSuccess) return e;
        const int t = h[0], done = h[2];
        if (done) break;
        if (launched > c.k) return cudaErrorLaunchFailure;   // no progress: cannot happen with u < 1
        need = (c.k - t + B - 1) / B;
    }
    const size_t tot = (size_t)c.k * c.d;
    const int ggrid = (int)std::max<size_t>(1, std::min<size_t>((size_t)c.num_sms * 4, (tot + 255) / 256));
    rs_gather_kernel<<<ggrid, 256, 0, c.stream>>>(c.C, c.d, c.chosen, c.k, centers);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace kmp
