// recluster_lloyd.cu -- Alg. 2 step 7 (candidate weights), step 8 (weighted
// k-means++, Alg. 1 with multiplicities, Sec. 4.2) and the centroid half of
// Lloyd's iteration (Sec. 3.1 centroid, Sec. 1 local search).
//
// The centroid update is a segmented sum: labels are counting-sorted into a
// stable permutation (per-block histograms, a column scan, one warp per block
// scattering in point order), then one CTA per cluster sums its members' rows in
// FP64 in a fixed order.  Results do not depend on scheduling.
#include <float.h>

#include <algorithm>
#include <cstdlib>

#include "dfloat.cuh"
#include "kmpar_internal.cuh"

namespace kmp {

// ------------------------------------------------------------------ step 7
__global__ void weights_kernel(const int32_t *__restrict__ idx, int64_t n, long long *w) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(reinterpret_cast<unsigned long long *>(w) + idx[i], 1ull);
}

cudaError_t launch_weights(Ctx &c) {
    cudaError_t e = cudaMemsetAsync(c.w, 0, sizeof(long long) * c.cap_total, c.stream);
    if (e != cudaSuccess) return e;
    weights_kernel<<<c.num_sms * 8, 256, 0, c.stream>>>(c.idx, c.n, c.w);
    count_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ step 8
// Weighted k-means++ (Alg. 1 with multiplicities w): k sequential draws over the m
// candidates.  One cooperative launch, one CTA of 704 threads per SM; the
// candidates are cut into fixed chunks of 32 (FP64 shuffle scans) and CTA b owns
// the contiguous chunk range [b cpc, (b+1) cpc); its warps 1.. take its chunks in
// phases A and C, warp 0 takes phase B.  Per draw t:
//   A  each warp: masses e_j = w_j (t = 0) or w_j D^2_j, inclusive warp scan;
//      chunk totals -> gchunk; the CTA's total (its chunks in a fixed order) is
//      published, after a fence, as one word tagged with the draw
//   B  CTA 0 (warp 0) waits until all G words carry the draw's tag (this wait is
//      the draw's grid barrier), then finds the pick from the totals: a fixed-order
//      prefix over the CTA totals gives the owning CTA of the target u_t * total, a
//      prefix over that CTA's chunk totals the chunk, a scan of the chunk's masses
//      the first candidate whose prefix exceeds the target; it publishes the pick
//      as one tagged word, which one lane of every other CTA polls
//   C  every warp: D^2_j <- min(D^2_j, ||c_j - c_pick||^2) in the exact FP32 form,
//      reading the candidates from a transposed copy (coordinate-major), so a
//      warp's 32 candidates are one coalesced 128-byte load per coordinate.
// The D^2 values in global memory (read in B for the picked chunk) and the chunk
// totals alternate between two buffers by the parity of the draw: a CTA can only
// write draw t + 2's values after every CTA has published draw t + 1, that is after
// every CTA has finished reading draw t's.  One wait per draw, bounded by `wait`
// clock cycles (about 2 s by default): a timeout raises the error word and every CTA
// returns.
constexpr int kRcThreads = 704;   // 21 chunk workers + the pick warp; 88 registers a thread
constexpr int kRcPre = 16;        // global coordinates per lane loaded while the pick is found
constexpr int kRcLaneWords = 8;   // CTA totals per lane of warp 0: G <= 256
constexpr unsigned long long kRcWait = 4000000000ull;

struct RcSync {
    int abort;   // set by the CTA whose wait ran out; the others return
};

// A CTA's total of one draw is published as one 64-bit word: the FP64 bits with
// the low 8 mantissa bits replaced by a tag of the draw (0x80 | (t >> 1) & 0x7f,
// never 0, and different for draws t and t - 2, which share a buffer).  A reader
// polls the word until the tag is its draw's; the value is then the word with the
// tag bits cleared (the total truncated by at most 2^-44 of itself, the same value
// in every CTA).
__device__ __forceinline__ unsigned long long rc_tag(int step) {
    return 0x80ull | ((unsigned long long)(step >> 1) & 0x7full);
}
__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

__device__ __forceinline__ double warp_incl_scan_f64(double v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Masses and prefix sums of the grid form are double floats (dfloat.cuh): the picks
// they give can differ from exact arithmetic only inside the near-tie window that
// flags a draw.

// weights as two floats whose sum is exact (w < 2^48)
__global__ void weight_split_kernel(const long long *__restrict__ w, const DevState *st, float2 *__restrict__ wf2) {
    const int m = st->m;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) wf2[j] = weight_split(w[j]);
}

// candidates (m x d, row-major) -> CT (d x mp, coordinate-major), 32 x 32 tiles
__global__ void transpose_cand_kernel(const float *__restrict__ C, int d, const DevState *st, int mp,
                                      float *__restrict__ CT) {
    __shared__ float tile[32][33];
    const int m = st->m;
    const int j0 = blockIdx.x * 32, q0 = blockIdx.y * 32;
    if (j0 >= m) return;
    for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
        const int j = j0 + ty, q = q0 + threadIdx.x;
        tile[ty][threadIdx.x] = (j < m && q < d) ? C[(int64_t)j * d + q] : 0.f;
    }
    __syncthreads();
    for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
        const int q = q0 + ty, j = j0 + threadIdx.x;
        if (q < d && j < m) CT[(int64_t)q * mp + j] = tile[threadIdx.x][ty];
    }
}

// Lane-parallel search of a fixed-order prefix: values v[lo .. hi) (global, read
// past L1), lane l summing its consecutive share; returns the first index whose
// running prefix (starting at `start`) exceeds target (-1: none) and the prefix
// before it.  Every CTA gets the same answer from the same values.
__device__ __forceinline__ int prefix_find(const double *v, int lo, int hi, double start, double target, int lane,
                                           double *before, double *total_out) {
    const int cnt = hi - lo;
    const int q = (cnt + 31) / 32;
    const int a = lo + min(cnt, lane * q), b = lo + min(cnt, lane * q + q);
    double ls = 0.0;
    for (int i = a; i < b; ++i) ls += __ldcg(v + i);
    const double incl = warp_incl_scan_f64(ls, lane);
    double excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0.0;
    if (total_out) *total_out = start + __shfl_sync(0xffffffffu, incl, 31);
    int hit = -1;
    double bf = 0.0, run = start + excl;
    for (int i = a; i < b; ++i) {
        const double pre = run;
        run = run + __ldcg(v + i);
        if (run > target) { hit = i; bf = pre; break; }
    }
    const unsigned any = __ballot_sync(0xffffffffu, hit >= 0);
    if (!any) return -1;
    const int src = __ffs(any) - 1;
    *before = __shfl_sync(0xffffffffu, bf, src);
    return __shfl_sync(0xffffffffu, hit, src);
}

// prefix_find with the values cached in registers (at most 8 per lane): one pass
// over global memory for the sum, the scan and the search
__device__ __forceinline__ int prefix_find_reg(const double *v, int lo, int hi, double start, double target, int lane,
                                               double *before, double *total_out) {
    const int cnt = hi - lo;
    const int q = (cnt + 31) / 32;
    if (q > 8) return prefix_find(v, lo, hi, start, target, lane, before, total_out);
    const int a = lo + min(cnt, lane * q), b = lo + min(cnt, lane * q + q);
    double vals[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) vals[t] = (t < q && a + t < b) ? __ldcg(v + a + t) : 0.0;
    double ls = 0.0;
#pragma unroll
    for (int t = 0; t < 8; ++t)
        if (t < q && a + t < b) ls += vals[t];
    const double incl = warp_incl_scan_f64(ls, lane);
    double excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0.0;
    if (total_out) *total_out = start + __shfl_sync(0xffffffffu, incl, 31);
    int hit = -1;
    double bf = 0.0, run = start + excl;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        if (hit < 0 && t < q && a + t < b) {
            const double pre = run;
            run = run + vals[t];
            if (run > target) { hit = a + t; bf = pre; }
        }
    }
    const unsigned any = __ballot_sync(0xffffffffu, hit >= 0);
    if (!any) return -1;
    const int src = __ffs(any) - 1;
    *before = __shfl_sync(0xffffffffu, bf, src);
    return __shfl_sync(0xffffffffu, hit, src);
}

// last index in [lo, hi) with a positive value (-1: none)
__device__ __forceinline__ int last_positive(const double *v, int lo, int hi, int lane) {
    int best = -1;
    for (int i = lo + lane; i < hi; i += 32)
        if (__ldcg(v + i) > 0.0) best = i;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    return best;
}

__global__ void __launch_bounds__(kRcThreads, 1) recluster_kernel(
    const float *__restrict__ C, const float *__restrict__ CT, int mp, const float2 *__restrict__ wf2, DevState *st,
    int d, int k, uint64_t seed, float *rD2buf, int32_t *chosen, float *centers, double *gchunk, int nchunk_cap,
    unsigned long long *slots, int cpc_cap, int qs, RcSync *sync, int *err, unsigned long long wait) {
    // shared: cpc_cap chunk totals, the CTA's candidates' weights (FP64) and D^2,
    // d floats of the pick's row, then the first qs coordinates of the CTA's
    // candidates (coordinate-major, staged once: they do not change across draws)
    extern __shared__ double rsm[];
    double *ctl = rsm;
    double *wl = rsm + cpc_cap;
    float2 *wl2 = reinterpret_cast<float2 *>(wl);   // the weights as two floats (8 bytes each)
    float *dl = reinterpret_cast<float *>(wl + (size_t)cpc_cap * 32);
    float *cnew = dl + (size_t)cpc_cap * 32;
    float *cts = cnew + ((d + 31) & ~31);
    __shared__ int s_pick, s_near, s_done, s_abort;
    __shared__ double s_tot, s_tgt, s_preb, s_prec;   // CTA 0: the draw's total, target and prefixes
    __shared__ int s_ob, s_nearL, s_chr;               // CTA 0: owning CTA, its fallback flag, chunk
    const int m = st->m;
    const int nchunk = (m + 31) / 32;
    const int G = gridDim.x;
    const int cpc = (nchunk + G - 1) / G;
    const int b = blockIdx.x;
    const int c0 = min(nchunk, b * cpc), c1 = min(nchunk, c0 + cpc);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = kRcThreads / 32;
    const int nl = (c1 - c0) * 32;   // the CTA's candidate slots
    const int qg = (G + 31) / 32;   // CTA totals read per lane of warp 0 (G <= 32 kRcLaneWords)
    const int ga = min(G, lane * qg), gb = min(G, lane * qg + qg);
    for (int ch = c0 + wid; ch < c1; ch += nwarps) {
        const int j = ch * 32 + lane;
        wl2[(ch - c0) * 32 + lane] = j < m ? wf2[j] : make_float2(0.f, 0.f);
    }
    for (int f = threadIdx.x; f < qs * nl; f += kRcThreads) {
        const int q = f / nl, jl = f - q * nl;
        const int j = c0 * 32 + jl;
        cts[(size_t)q * nl + jl] = j < m ? CT[(int64_t)q * mp + j] : 0.f;
    }
    __syncthreads();

    for (int step = 0; step < k; ++step) {
        double *gch = gchunk + (size_t)(step & 1) * nchunk_cap;
        unsigned long long *gs = slots + (size_t)(step & 1) * G;
        const unsigned long long tag = rc_tag(step);
        const float *rD2prev = rD2buf + (size_t)((step + 1) & 1) * mp;   // D^2 after draw step - 1
        float *rD2 = rD2buf + (size_t)(step & 1) * mp;
        // ---- A (warps 1..): chunk masses and the CTA total.  A chunk is scanned by
        // the warp that updates its D^2 in phase C, so its D^2 values in shared
        // memory pass between phases within one warp
        for (int ch = c0 + wid - 1; wid > 0 && ch < c1; ch += nwarps - 1) {
            const int j = ch * 32 + lane;
            const int jl = (ch - c0) * 32 + lane;
            Df e = {0.f, 0.f};
            if (j < m) e = df_mass(wl2[jl], dl[jl], step == 0);
            const Df incl = warp_incl_scan_df(e, lane);
            if (lane == 31) {
                const double tot = df_to_double(incl);
                ctl[ch - c0] = tot;
                gch[ch] = tot;
            }
        }
        __threadfence();   // every thread's chunk totals (and last draw's D^2) before the flag
        __syncthreads();
        if (wid == 0) {
            double s = 0.0;
            for (int i = lane; i < c1 - c0; i += 32) s += ctl[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) {
                *reinterpret_cast<volatile unsigned long long *>(gs + b) =
                    (__double_as_longlong(s) & ~0xffull) | tag;
            }
        }
        // ---- B, CTA 0 (warp 0): wait until every CTA's word carries this draw's tag
        // (the words of all G CTAs are polled together, so the wait ends one load
        // after the last CTA publishes), find the pick and publish it as one tagged
        // word; the other CTAs (one lane) poll that word.  One CTA reads the published
        // totals and the owning chunk: no contention of G CTAs on the same lines.
        unsigned long long *pw = slots + 2 * (size_t)G + (step & 1);
        // With at most one owned chunk per worker warp, CTA 0's worker warps fetch the
        // owning CTA's masses (one chunk each, one round trip) while warp 0 waits, and
        // the chunk and candidate are found from them; otherwise warp 0 reads the
        // owner's published chunk totals and then the chunk's masses.
        const bool par = cpc <= nwarps - 1;
        if (b == 0) {
        if (wid == 0) {
            unsigned long long gw[kRcLaneWords];
            int ok = 1;
            const unsigned long long t0 = clock64();
            for (;;) {
                bool mine = true;
#pragma unroll
                for (int t = 0; t < kRcLaneWords; ++t) {
                    if (t < qg && ga + t < gb) {
                        gw[t] = ld_volatile_u64(gs + ga + t);
                        mine = mine && (gw[t] & 0xffull) == tag;
                    }
                }
                if (__all_sync(0xffffffffu, mine)) break;
                int stop = 0;
                if (lane == 0) {
                    if (*(volatile int *)&sync->abort) stop = 1;
                    else if (clock64() - t0 > wait) {
                        atomicCAS(err, 0, 1);
                        atomicExch(&sync->abort, 1);
                        stop = 1;
                    }
                }
                if (__shfl_sync(0xffffffffu, stop, 0)) { ok = 0; break; }
            }
            __threadfence();   // the chunk totals and D^2 the words were published after
            double total = 0.0, before = 0.0;
            int pick = -1, near = 0;
            double gv[kRcLaneWords];
#pragma unroll
            for (int t = 0; t < kRcLaneWords; ++t)
                gv[t] = (ok && t < qg && ga + t < gb) ? __longlong_as_double((long long)(gw[t] & ~0xffull)) : 0.0;
            const double u = uniform53((uint64_t)step, 0, TAG_RECLUSTER, seed);
            // the total first (the target depends on it): a sum with the same association
            // as the search below
            double ls = 0.0;
#pragma unroll
            for (int t = 0; t < kRcLaneWords; ++t)
                if (t < qg && ga + t < gb) ls += gv[t];
            const double gincl = warp_incl_scan_f64(ls, lane);
            total = __shfl_sync(0xffffffffu, gincl, 31);
            if (total > 0.0) {
                const double target = __dmul_rn(u, total);
                double gex = __shfl_up_sync(0xffffffffu, gincl, 1);
                if (lane == 0) gex = 0.0;
                int hit = -1;
                double bf = 0.0, run = gex;
#pragma unroll
                for (int t = 0; t < kRcLaneWords; ++t) {
                    if (hit < 0 && t < qg && ga + t < gb) {
                        const double pre = run;
                        run = run + gv[t];
                        if (run > target) { hit = ga + t; bf = pre; }
                    }
                }
                const unsigned anyb = __ballot_sync(0xffffffffu, hit >= 0);
                int ob = -1;
                if (anyb) {
                    const int src = __ffs(anyb) - 1;
                    before = __shfl_sync(0xffffffffu, bf, src);
                    ob = __shfl_sync(0xffffffffu, hit, src);
                }
                double pre_b = before;
                if (ob < 0) {   // rounding left the target at the end: the last CTA with mass
                    int lb = -1;
#pragma unroll
                    for (int t = 0; t < kRcLaneWords; ++t)
                        if (t < qg && ga + t < gb && gv[t] > 0.0) lb = ga + t;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) lb = max(lb, __shfl_xor_sync(0xffffffffu, lb, o));
                    ob = lb;
                    pre_b = 0.0;
                    near = 1;
                }
                if (par) {
                    if (lane == 0) { s_tgt = target; s_preb = pre_b; s_ob = ob; s_nearL = near; }
                } else {
                const int oc0 = min(nchunk, ob * cpc), oc1 = min(nchunk, oc0 + cpc);
                int ch = near ? -1 : prefix_find_reg(gch, oc0, oc1, pre_b, target, lane, &before, nullptr);
                double pre_c = before;
                if (ch < 0) { ch = last_positive(gch, oc0, oc1, lane); near = 1; }
                const int j = ch * 32 + lane;
                Df ef = {0.f, 0.f};
                if (j < m) ef = df_mass(wf2[j], __ldcg(rD2prev + j), step == 0);
                const Df inclf = warp_incl_scan_df(ef, lane);
                const double e = df_to_double(ef), incl = df_to_double(inclf);
                const unsigned pos = __ballot_sync(0xffffffffu, j < m && e > 0.0);
                if (!near) {
                    const double cum = pre_c + incl, cum0 = pre_c + (incl - e);
                    const unsigned hit = __ballot_sync(0xffffffffu, j < m && cum > target);
                    if (hit) {
                        const int hl = __ffs(hit) - 1;
                        pick = ch * 32 + hl;
                        const int nr = fabs(target - cum0) <= 1e-6 * total || fabs(cum - target) <= 1e-6 * total;
                        near = __shfl_sync(0xffffffffu, nr, hl);
                    } else {
                        near = 1;
                    }
                }
                if (pick < 0) pick = ch * 32 + 31 - __clz(pos);   // last positive mass of the chunk
                }
            }
            if (lane == 0) {
                s_tot = total;
                s_done = !(total > 0.0);
                s_abort = !ok;
                // the pick is published here unless the worker warps take part in it
                if (!par || !(total > 0.0) || !ok) {
                    s_pick = pick;
                    s_near = near;
                    if (ok)
                        *reinterpret_cast<volatile unsigned long long *>(pw) =
                            ((unsigned long long)(uint32_t)max(pick, 0) << 32) | ((unsigned long long)near << 8) |
                            ((unsigned long long)(total > 0.0 ? 0 : 1) << 9) | tag;
                }
            }
        }
        if (par) {
            __syncthreads();
            const bool go = !s_abort && s_tot > 0.0;
            const int ob = go ? s_ob : 0;
            const int oc0 = min(nchunk, ob * cpc), oc1 = min(nchunk, oc0 + cpc);
            // worker warp w: the masses of the owner's chunk oc0 + w - 1 and their scan
            // (the same FP64 products and association as the owner's own scan)
            const int chw = oc0 + wid - 1;
            const int jw = chw * 32 + lane;
            double e = 0.0, incl = 0.0;
            if (go && wid > 0 && chw < oc1) {
                Df ef = {0.f, 0.f};
                if (jw < m) ef = df_mass(wf2[jw], __ldcg(rD2prev + jw), step == 0);
                const Df inclf = warp_incl_scan_df(ef, lane);
                incl = df_to_double(inclf);
                e = df_to_double(ef);
                if (lane == 31) ctl[wid - 1] = incl;
            }
            __syncthreads();
            if (go && wid == 0) {
                // the chunk: a fixed-order prefix over the owner's chunk totals from the
                // prefix before the owner (as the search over published chunk totals)
                const int cnt = oc1 - oc0;
                const double val = lane < cnt ? ctl[lane] : 0.0;
                const double vin = warp_incl_scan_f64(val, lane);
                double ex = __shfl_up_sync(0xffffffffu, vin, 1);
                if (lane == 0) ex = 0.0;
                const double pre = s_preb + ex;
                const double run = pre + val;
                int nearc = s_nearL;
                const unsigned hitm = nearc ? 0u : __ballot_sync(0xffffffffu, lane < cnt && run > s_tgt);
                int chr;
                double prec = 0.0;
                if (hitm) {
                    chr = __ffs(hitm) - 1;
                    prec = __shfl_sync(0xffffffffu, pre, chr);
                } else {   // the last chunk with mass
                    const unsigned posm = __ballot_sync(0xffffffffu, lane < cnt && val > 0.0);
                    chr = posm ? 31 - __clz(posm) : 0;
                    nearc = 1;
                }
                if (lane == 0) { s_chr = chr; s_prec = prec; s_nearL = nearc; }
            }
            __syncthreads();
            if (go && wid == s_chr + 1) {
                // the candidate, from this warp's masses
                const double target = s_tgt, total = s_tot, pre_c = s_prec;
                int near = s_nearL, pick = -1;
                const unsigned pos = __ballot_sync(0xffffffffu, jw < m && e > 0.0);
                if (!near) {
                    const double cum = pre_c + incl, cum0 = pre_c + (incl - e);
                    const unsigned hit = __ballot_sync(0xffffffffu, jw < m && cum > target);
                    if (hit) {
                        const int hl = __ffs(hit) - 1;
                        pick = chw * 32 + hl;
                        const int nr = fabs(target - cum0) <= 1e-6 * total || fabs(cum - target) <= 1e-6 * total;
                        near = __shfl_sync(0xffffffffu, nr, hl);
                    } else {
                        near = 1;
                    }
                }
                if (pick < 0) pick = chw * 32 + 31 - __clz(pos);   // last positive mass of the chunk
                if (lane == 0) {
                    s_pick = pick;
                    s_near = near;
                    *reinterpret_cast<volatile unsigned long long *>(pw) =
                        ((unsigned long long)(uint32_t)pick << 32) | ((unsigned long long)near << 8) | tag;
                }
            }
        }
        } else if (wid == 0 && lane == 0) {
            int ok = 1;
            unsigned long long v;
            const unsigned long long t0 = clock64();
            for (;;) {
                v = ld_volatile_u64(pw);
                if ((v & 0xffull) == tag) break;
                if (*(volatile int *)&sync->abort) { ok = 0; break; }
                if (clock64() - t0 > wait) {
                    atomicCAS(err, 0, 1);
                    atomicExch(&sync->abort, 1);
                    ok = 0;
                    break;
                }
            }
            s_pick = (int)(v >> 32);
            s_near = (int)((v >> 8) & 1);
            s_done = (int)((v >> 9) & 1);
            s_abort = !ok;
        }
        // warps 1.. load the first global coordinates of their first chunk while the
        // pick is found (they do not depend on it)
        float pre[kRcPre];
        const int chp = c0 + wid - 1;
        const int np = (wid > 0 && chp < c1) ? max(0, min(kRcPre, d - qs)) : 0;
        {
            const int jp = min(chp * 32 + lane, m - 1);
#pragma unroll
            for (int u2 = 0; u2 < kRcPre; ++u2) pre[u2] = u2 < np ? __ldg(CT + (int64_t)(qs + u2) * mp + jp) : 0.f;
        }
        __syncthreads();
        if (s_abort) return;
        if (s_done) {
            // positive mass exhausted: the remaining draws repeat the first center
            if (b == 0) {
                for (int s2 = step + threadIdx.x; s2 < k; s2 += kRcThreads) chosen[s2] = step > 0 ? chosen[0] : 0;
                if (threadIdx.x == 0) st->warn = 1;
                __syncthreads();
                const int src = step > 0 ? chosen[0] : 0;
                for (int s2 = step; s2 < k; ++s2)
                    for (int qq = threadIdx.x; qq < d; qq += kRcThreads)
                        centers[(int64_t)s2 * d + qq] = C[(int64_t)src * d + qq];
            }
            return;
        }
        const int pick = s_pick;
        if (b == 0 && threadIdx.x == 0) {
            chosen[step] = pick;
            if (s_near) atomicAdd(&st->recluster_near, 1ull);
        }
        for (int qq = threadIdx.x; qq < d; qq += kRcThreads) {
            const float v = __ldcg(C + (int64_t)pick * d + qq);
            cnew[qq] = v;
            if (b == 0) centers[(int64_t)step * d + qq] = v;
        }
        __syncthreads();
        // ---- C (warps 1..): D^2 update of own candidates (t = x_q - c_q, fma, q
        // ascending): the first qs coordinates from shared memory, the rest from the
        // transposed copy, 32 loads issued before their FMA chain runs
        // A candidate's squared distance is a sum of non-negative terms added in a
        // fixed order, so its FP32 partial sums never decrease: once every lane's
        // partial sum has reached its D^2 (a warp vote every 16 coordinates), no D^2
        // of the warp can change and the rest of the sum is skipped.  Most
        // candidates are far from the new center, so most warps stop within the
        // coordinates held in shared memory.
        auto update = [&](int ch, bool first) {
            const int j = ch * 32 + lane;
            const int jl = (ch - c0) * 32 + lane;
            const bool act = j < m;
            const float lim = (step == 0 || !act) ? __uint_as_float(0x7f800000u) : dl[jl];
            float v = 0.f;
            const float *col = CT + (act ? j : 0);
            int q = 0;
            bool settled = false;
            while (q < qs && !settled) {
                const int qe = min(qs, q + 16);
                for (; q < qe; ++q) {
                    const float t = __fsub_rn(cts[(size_t)q * nl + jl], cnew[q]);
                    v = __fmaf_rn(t, t, v);
                }
                settled = __all_sync(0xffffffffu, !act || v >= lim);
            }
            // the remaining coordinates from the transposed copy: those loaded ahead,
            // then batches of up to 32 loads issued together, each followed by its FMA
            // chain in order
            if (first && !settled && np > 0) {
#pragma unroll
                for (int u2 = 0; u2 < kRcPre; ++u2) {
                    if (u2 < np) {
                        const float t = __fsub_rn(pre[u2], cnew[q + u2]);
                        v = __fmaf_rn(t, t, v);
                    }
                }
                q += np;
                settled = __all_sync(0xffffffffu, !act || v >= lim);
            }
            while (q < d && !settled) {
                const int nb = min(32, d - q);
                float buf[32];
#pragma unroll
                for (int u2 = 0; u2 < 32; ++u2) buf[u2] = (act && u2 < nb) ? __ldg(col + (int64_t)(q + u2) * mp) : 0.f;
#pragma unroll
                for (int u2 = 0; u2 < 32; ++u2) {
                    if (u2 < nb) {
                        const float t = __fsub_rn(buf[u2], cnew[q + u2]);
                        v = __fmaf_rn(t, t, v);
                    }
                }
                q += nb;
                settled = __all_sync(0xffffffffu, !act || v >= lim);
            }
            if (!act) return;
            // a settled partial sum is >= D^2, so the minimum keeps D^2 as the full sum would
            const float nv = step == 0 ? v : fminf(dl[jl], v);
            dl[jl] = nv;
            rD2[j] = nv;
        };
        if (wid > 0 && chp < c1) {
            update(chp, true);
            for (int ch = chp + nwarps - 1; ch < c1; ch += nwarps - 1) update(ch, false);
        }
        // the next draw's flags order these writes before any CTA reads them
    }
}

// ------------------------------------------------------------------ step 8, one cluster
// The same draws for candidate sets whose rows fit the shared memory of one
// thread-block cluster (kClSize CTAs of 1024 threads).  CTA r owns the fixed
// chunk range [r cpc, (r+1) cpc) of 32-candidate chunks and keeps their rows,
// weights and D^2 in its shared memory.  Per draw:
//   A  warp scans of the masses of the CTA's chunks, the CTA total (chunks in
//      order)                                             ... cluster barrier
//   B  every CTA reads the CTA totals over distributed shared memory in rank
//      order (FP64): total, target u_t * total, the owning CTA; the owner finds
//      the chunk and the candidate as recluster_kernel does (same near-tie and
//      rounding rules) and writes the pick into every CTA   ... cluster barrier
//   C  every CTA: D^2_j <- min(D^2_j, ||c_j - c_pick||^2) for its candidates.
// Hardware cluster barriers replace the grid barrier and the published flag;
// every CTA takes the same branches (the totals it reads are the same), so all
// of them reach every barrier.
constexpr int kClSize = 8;
constexpr int kClThreads = 1024;

__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cl_map(const void *p, uint32_t rank) {
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(a)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return a;
}
__device__ __forceinline__ double cl_ld_f64(uint32_t a) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void cl_st_s32(uint32_t a, int v) {
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// shared memory of one CTA: chunk totals, the picked row, D^2, weights (FP64), rows
// (stride cl_stride(d): 8-byte aligned, conflict-free lane-per-row reads)
__host__ __device__ __forceinline__ int cl_stride(int d) { return (d & 1) ? d : d + ((6 - (d & 3)) & 3); }
__host__ __device__ __forceinline__ size_t cl_smem_bytes(int cpc, int d, bool rows) {
    const size_t dp = (size_t)((d + 3) & ~3);
    return sizeof(double) * cpc + sizeof(float) * dp + sizeof(float) * 32 * (size_t)cpc +
           sizeof(double) * 32 * (size_t)cpc + (rows ? sizeof(float) * 32 * (size_t)cpc * cl_stride(d) : 0) +
           sizeof(int) * (size_t)cpc;
}

// exact FP32 difference form of a row in shared memory (8-byte loads for even d),
// stopping once its partial sum reaches lim: the partial sums of non-negative terms
// never decrease, so a returned value >= lim means the full sum is >= lim too (the
// caller only needs to know whether it is below lim)
__device__ __forceinline__ float cl_dist2_lim(const float *x, const float *c, int d, float lim) {
    float s = 0.f;
    if ((d & 1) == 0) {
        const float2 *x2 = reinterpret_cast<const float2 *>(x), *c2 = reinterpret_cast<const float2 *>(c);
        for (int p0 = 0; p0 < (d >> 1); p0 += 8) {
            const int pe = min(d >> 1, p0 + 8);
            for (int p = p0; p < pe; ++p) {
                const float2 a = x2[p], b = c2[p];
                float t = __fsub_rn(a.x, b.x);
                s = __fmaf_rn(t, t, s);
                t = __fsub_rn(a.y, b.y);
                s = __fmaf_rn(t, t, s);
            }
            if (s >= lim) return s;
        }
    } else {
        for (int q0 = 0; q0 < d; q0 += 16) {
            const int qe = min(d, q0 + 16);
            for (int q = q0; q < qe; ++q) {
                const float t = __fsub_rn(x[q], c[q]);
                s = __fmaf_rn(t, t, s);
            }
            if (s >= lim) return s;
        }
    }
    return s;
}
__device__ __forceinline__ float dist2_fp32_lim(const float *__restrict__ x, const float *__restrict__ c, int d,
                                                float lim) {
    float s = 0.f;
    for (int q0 = 0; q0 < d; q0 += 16) {
        const int qe = min(d, q0 + 16);
        for (int q = q0; q < qe; ++q) {
            const float t = __fsub_rn(x[q], c[q]);
            s = __fmaf_rn(t, t, s);
        }
        if (s >= lim) return s;
    }
    return s;
}

// FP64 sum of v[0..n) by one warp in a fixed order: lane l adds v[l], v[l + 32],
// ... in order, then a fixed butterfly; every lane gets the total
__device__ __forceinline__ double warp_sum_fixed(const double *v, int n, int lane) {
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

__global__ void __launch_bounds__(kClThreads, 1)
    recluster_cluster_kernel(const float *__restrict__ C, const long long *__restrict__ w, DevState *st, int d, int k,
                             uint64_t seed, int cpc_cap, int rows_in_smem, int32_t *chosen, float *centers) {
    extern __shared__ __align__(16) unsigned char csm[];
    double *cm = reinterpret_cast<double *>(csm);                       // chunk totals
    float *cnew = reinterpret_cast<float *>(cm + cpc_cap);               // picked row
    float *rd2 = cnew + ((d + 3) & ~3);                                  // D^2 of own candidates
    double *wl = reinterpret_cast<double *>(rd2 + 32 * cpc_cap);         // weights
    float *crow = reinterpret_cast<float *>(wl + 32 * cpc_cap);          // rows (rows_in_smem)
    // per chunk: some D^2 fell in the last draw, so its masses must be scanned again
    int *dirty = reinterpret_cast<int *>(crow + (rows_in_smem ? 32 * (size_t)cpc_cap * cl_stride(d) : 0));
    __shared__ double s_ctot, s_pre, s_total, s_target;
    __shared__ int s_pick, s_owner, s_miss;
    const int rank = (int)cl_rank();
    const int t_id = threadIdx.x, lane = t_id & 31, wid = t_id >> 5;
    const int m = st->m;
    const int nchunk = (m + 31) / 32;
    const int cpc = min(cpc_cap, (nchunk + kClSize - 1) / kClSize);   // balanced over the CTAs
    const int c0 = min(nchunk, rank * cpc), c1 = min(nchunk, c0 + cpc);
    const int nc = c1 - c0;
    const int j0 = c0 * 32, j1 = min(m, c1 * 32);
    const int rs = rows_in_smem ? cl_stride(d) : d;
    for (int j = j0 + t_id; j < j1; j += kClThreads) wl[j - j0] = (double)w[j];
    if (rows_in_smem)
        for (int f = t_id; f < (j1 - j0) * d; f += kClThreads) {
            const int jr = f / d, q = f - jr * d;
            crow[jr * rs + q] = C[(int64_t)j0 * d + f];
        }
    const float *rows = rows_in_smem ? crow : C + (int64_t)j0 * d;
    for (int i = t_id; i < cpc_cap; i += kClThreads) dirty[i] = 1;
    __syncthreads();
    for (int step = 0; step < k; ++step) {
        // ---- A: chunk masses and the CTA total.  A chunk none of whose D^2 fell in
        // the last draw keeps its total: rescanning it would give the same value.
        for (int ch = c0 + wid; ch < c1; ch += kClThreads / 32) {
            if (!dirty[ch - c0]) continue;   // uniform per warp
            const int j = ch * 32 + lane;
            double e = 0.0;
            if (j < m) e = step == 0 ? wl[j - j0] : __dmul_rn(wl[j - j0], (double)rd2[j - j0]);
            const double incl = warp_incl_scan_f64(e, lane);
            if (lane == 31) cm[ch - c0] = incl;
            __syncwarp();
            if (lane == 0) dirty[ch - c0] = 0;
        }
        __syncthreads();
        if (wid == 0) {
            const double s = warp_sum_fixed(cm, nc, lane);
            if (lane == 0) s_ctot = s;
        }
        cl_sync();
        // ---- B: totals in rank order, the owning CTA
        if (wid == 0) {
            const double v = lane < kClSize ? cl_ld_f64(cl_map(&s_ctot, lane)) : 0.0;
            const double pre = warp_incl_scan_f64(v, lane);
            const double total = __shfl_sync(0xffffffffu, pre, kClSize - 1);
            if (lane == 0) s_total = total;
            if (total > 0.0) {
                const double target = __dmul_rn(uniform53((uint64_t)step, 0, TAG_RECLUSTER, seed), total);
                // only CTAs with positive mass can own the draw (a scan prefix is not
                // monotone bit for bit, so the first prefix above the target could
                // otherwise belong to an empty CTA)
                const unsigned hit = __ballot_sync(0xffffffffu, lane < kClSize && v > 0.0 && pre > target);
                const unsigned pos = __ballot_sync(0xffffffffu, lane < kClSize && v > 0.0);
                const int owner = hit ? __ffs(hit) - 1 : 31 - __clz(pos);
                const double excl = __shfl_up_sync(0xffffffffu, pre, 1);   // exclusive prefix
                const double before = __shfl_sync(0xffffffffu, lane > 0 ? excl : 0.0, owner);
                if (lane == 0) {
                    s_target = target;
                    s_owner = owner;
                    s_miss = hit ? 0 : 1;
                    s_pre = before;
                }
            }
        }
        __syncthreads();
        const double total = s_total;
        if (!(total > 0.0)) {
            // positive mass exhausted: the remaining draws repeat the first center
            if (rank == 0) {
                for (int s = step + t_id; s < k; s += kClThreads) chosen[s] = step > 0 ? chosen[0] : 0;
                if (t_id == 0) st->warn = 1;
                __syncthreads();
                const int src = step > 0 ? chosen[0] : 0;
                for (int s = step; s < k; ++s)
                    for (int qq = t_id; qq < d; qq += kClThreads) centers[(int64_t)s * d + qq] = C[(int64_t)src * d + qq];
            }
            cl_sync();   // no CTA leaves while another may still read its shared memory
            return;
        }
        if (rank == s_owner && wid == 0) {
            const double target = s_target;
            bool miss = s_miss != 0;
            // the chunk whose running prefix first exceeds the target: chunk totals in
            // groups of 32, scanned in order (the last chunk with positive mass when
            // rounding hides the crossing)
            int ch = -1;
            double pre = 0.0, run = s_pre;
            for (int g0 = 0; g0 < nc && ch < 0 && !miss; g0 += 32) {
                const double v = g0 + lane < nc ? cm[g0 + lane] : 0.0;
                const double incl = run + warp_incl_scan_f64(v, lane);
                const unsigned hit = __ballot_sync(0xffffffffu, g0 + lane < nc && v > 0.0 && incl > target);
                if (hit) {
                    const int l = __ffs(hit) - 1;
                    ch = g0 + l;
                    pre = __shfl_sync(0xffffffffu, incl - v, l);
                }
                run = __shfl_sync(0xffffffffu, incl, 31);
            }
            if (ch < 0) {
                for (int g0 = ((nc - 1) / 32) * 32; g0 >= 0 && ch < 0; g0 -= 32) {
                    const unsigned pos = __ballot_sync(0xffffffffu, g0 + lane < nc && cm[g0 + lane] > 0.0);
                    if (pos) ch = g0 + 31 - __clz(pos);
                }
                miss = true;
            }
            const int chunk = c0 + ch;
            const int j = chunk * 32 + lane;
            double e = 0.0;
            if (j < m) e = step == 0 ? wl[j - j0] : __dmul_rn(wl[j - j0], (double)rd2[j - j0]);
            const double incl = warp_incl_scan_f64(e, lane);
            const double cum = pre + incl, cum0 = pre + (incl - e);
            const unsigned hit = miss ? 0u : __ballot_sync(0xffffffffu, j < m && e > 0.0 && cum > target);
            const unsigned pos = __ballot_sync(0xffffffffu, j < m && e > 0.0);   // nonzero: the chunk has mass
            const int pick = hit ? chunk * 32 + __ffs(hit) - 1 : chunk * 32 + 31 - __clz(pos);
            if (hit) {
                const bool near = fabs(target - cum0) <= 1e-6 * total || fabs(cum - target) <= 1e-6 * total;
                if (lane == __ffs(hit) - 1 && near) atomicAdd(&st->recluster_near, 1ull);
            } else if (lane == 0) {
                atomicAdd(&st->recluster_near, 1ull);
            }
            if (lane < kClSize) cl_st_s32(cl_map(&s_pick, lane), pick);
            if (lane == 0) chosen[step] = pick;
        }
        cl_sync();
        // ---- C: the picked row and the D^2 update
        const int pick = s_pick;
        for (int qq = t_id; qq < d; qq += kClThreads) {
            const float v = C[(int64_t)pick * d + qq];
            cnew[qq] = v;
            if (rank == 0) centers[(int64_t)step * d + qq] = v;
        }
        __syncthreads();
        // partial sums stop once they reach the candidate's D^2 (then no update)
        for (int j = j0 + t_id; j < j1; j += kClThreads) {
            const float lim = step == 0 ? __uint_as_float(0x7f800000u) : rd2[j - j0];
            const float v = rows_in_smem ? cl_dist2_lim(rows + (int64_t)(j - j0) * rs, cnew, d, lim)
                                         : dist2_fp32_lim(rows + (int64_t)(j - j0) * d, cnew, d, lim);
            if (step == 0 || v < rd2[j - j0]) {
                rd2[j - j0] = v;
                dirty[(j - j0) >> 5] = 1;
            }
        }
        __syncthreads();
    }
    cl_sync();   // no CTA leaves while another may still read its shared memory
}

// the cluster form applies when the largest candidate set's chunks fit the CTAs'
// shared memory (rows in shared memory when they fit too)
static bool cluster_plan(const Ctx &c, int *cpc, int *rows) {
    const int max_chunks = (c.cap_total + 31) / 32;
    *cpc = (max_chunks + kClSize - 1) / kClSize;
    const size_t budget = 200u * 1024u;
    *rows = cl_smem_bytes(*cpc, c.d, true) <= budget ? 1 : 0;
    return cl_smem_bytes(*cpc, c.d, false) <= budget && (size_t)c.cap_total * c.d <= (4u << 20);
}

cudaError_t launch_recluster_cluster(Ctx &c, float *centers, int cpc, int rows) {
    const size_t smem = cl_smem_bytes(cpc, c.d, rows != 0);
    cudaError_t e = cudaFuncSetAttribute(recluster_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClSize);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClSize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, recluster_cluster_kernel, (const float *)c.C, (const long long *)c.w, c.st, c.d,
                           c.k, c.seed, cpc, rows, c.chosen, centers);
    count_launches(1);
    return e;
}

size_t recluster_grid_floats(const Ctx &c) {
    int cpc = 0, rows = 0;
    const char *force_grid = std::getenv("KMPAR_RECLUSTER_GRID");
    const bool grid_only = force_grid && force_grid[0] == '1';
    if (!grid_only && cluster_plan(c, &cpc, &rows)) return 0;
    // the transposed candidates (d x mp) and the weights split into two floats (mp float2)
    return (size_t)((c.cap_total + 31) / 32) * 32 * (c.d + 2);
}

cudaError_t launch_transpose_cand(Ctx &c) {
    const int mp = (c.cap_total + 31) / 32 * 32;
    transpose_cand_kernel<<<dim3(mp / 32, (c.d + 31) / 32), dim3(32, 8), 0, c.stream>>>(c.C, c.d, c.st, mp, c.rCT);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_recluster(Ctx &c, float *centers) {
    cudaError_t e;
    int cpc = 0, rows = 0;
    // KMPAR_RECLUSTER_GRID=1 selects the cooperative grid form for every size (both
    // forms are tested against the oracle)
    const char *force_grid = std::getenv("KMPAR_RECLUSTER_GRID");
    const bool grid_only = force_grid && force_grid[0] == '1';
    if (!grid_only && cluster_plan(c, &cpc, &rows)) return launch_recluster_cluster(c, centers, cpc, rows);
    if (!c.rCT) return cudaErrorInvalidValue;   // kmpar_recluster allocates the transposed copy first
    if ((e = cudaMemsetAsync(c.rc_sync, 0, sizeof(RcSync), c.stream)) != cudaSuccess) return e;
    const int mp = (c.cap_total + 31) / 32 * 32;
    if ((e = launch_transpose_cand(c)) != cudaSuccess) return e;
    // one co-resident CTA per SM
    const int nchunk_cap = (c.cap_total + 31) / 32;
    int G = std::max(1, std::min(std::min(c.num_sms, 32 * kRcLaneWords), nchunk_cap));
    const int cpc_cap = (nchunk_cap + G - 1) / G;
    const size_t base_smem = sizeof(double) * (size_t)cpc_cap * 33 +
                             sizeof(float) * ((size_t)cpc_cap * 32 + (size_t)((c.d + 31) & ~31));
    int dev = 0, optin = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    const size_t budget = (size_t)optin - 1024;   // the kernel's static shared memory and slack
    if (base_smem > budget) return cudaErrorInvalidValue;   // beyond ~500,000 candidates per SM
    // as many leading coordinates of the CTA's candidates as fit
    int qs = (int)((budget - base_smem) / (sizeof(float) * (size_t)cpc_cap * 32));
    qs = std::max(0, std::min(qs, c.d));
    const size_t smem = base_smem + sizeof(float) * (size_t)qs * cpc_cap * 32;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(recluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, recluster_kernel, kRcThreads, smem)) !=
        cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    const float *Cp = c.C;
    const float *CTp = c.rCT;
    // weights as two floats each, after the transposed candidates
    const float2 *wp = reinterpret_cast<const float2 *>(c.rCT + (size_t)c.d * mp);
    weight_split_kernel<<<std::max(1, std::min(c.num_sms * 4, (mp + 255) / 256)), 256, 0, c.stream>>>(
        c.w, c.st, const_cast<float2 *>(wp));
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    DevState *stp = c.st;
    int d = c.d, k = c.k, mpv = mp, ncap = nchunk_cap, cpcv = cpc_cap, qsv = qs;
    uint64_t seed = c.seed;
    float *rD2 = c.rD2;
    int32_t *chosen = c.chosen;
    double *gch = c.rc_cmass;
    unsigned long long *slots = reinterpret_cast<unsigned long long *>(c.rc_cmass + 2 * (size_t)nchunk_cap);
    RcSync *sy = reinterpret_cast<RcSync *>(c.rc_sync);
    // words from an earlier call could carry this call's tags
    if ((e = cudaMemsetAsync(slots, 0, sizeof(unsigned long long) * (2 * (size_t)G + 2), c.stream)) != cudaSuccess)
        return e;
    int *err = c.rc_err;
    // KMPAR_WAIT_CYCLES bounds each per-draw wait (fault injection: a budget too short
    // for the CTAs to meet makes the call return KMPAR_ERR_TIMEOUT)
    unsigned long long wait = kRcWait;
    if (const char *wv = std::getenv("KMPAR_WAIT_CYCLES")) {
        char *end = nullptr;
        const unsigned long long x = std::strtoull(wv, &end, 10);
        if (end && *end == 0 && *wv) wait = x;
    }
    void *args[] = {&Cp, &CTp, &mpv, &wp, &stp, &d, &k, &seed, &rD2, &chosen, &centers, &gch, &ncap, &slots, &cpcv,
                    &qsv, &sy, &err, &wait};
    e = cudaLaunchCooperativeKernel((const void *)recluster_kernel, dim3(G), dim3(kRcThreads), args, smem, c.stream);
    count_launches(1);
    return e;
}

size_t recluster_sync_bytes() { return sizeof(RcSync); }

// ------------------------------------------------------------------ step 8 alternative
// Lloyd's iteration on the weighted candidates: the centroid half.  One block per
// center j: the block walks the candidate labels in chunks of its size, keeps the
// members of j in ascending order (ordered block compaction) and thread q adds
// w_c * c_q in FP64 (rounded product, then rounded sum, as the definition is
// written); the center becomes the FP64 quotient by sum w_c rounded to FP32, or
// keeps its place when no candidate is its nearest.
constexpr int kWlThreads = 256;
constexpr int kWlMaxQ = 16;   // d <= 16 * kWlThreads

__global__ void __launch_bounds__(kWlThreads) weighted_centroid_kernel(const float *__restrict__ cand,
                                                                       const long long *__restrict__ w,
                                                                       const int32_t *__restrict__ lab, int m, int d,
                                                                       float *__restrict__ centers) {
    __shared__ int mem[kWlThreads];
    __shared__ int wcnt[kWlThreads / 32];
    const int j = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    double acc[kWlMaxQ];
#pragma unroll
    for (int u = 0; u < kWlMaxQ; ++u) acc[u] = 0.0;
    long long wsum = 0;
    for (int base = 0; base < m; base += kWlThreads) {
        const int i = base + tid;
        const bool mine = i < m && lab[i] == j;
        const unsigned mask = __ballot_sync(0xffffffffu, mine);
        if (lane == 0) wcnt[wid] = __popc(mask);
        __syncthreads();
        int before = 0, tot = 0;
        for (int q = 0; q < kWlThreads / 32; ++q) {
            if (q < wid) before += wcnt[q];
            tot += wcnt[q];
        }
        if (mine) mem[before + __popc(mask & ((1u << lane) - 1u))] = i;
        __syncthreads();
        for (int t = 0; t < tot; ++t) {
            const int c = mem[t];
            const double wc = (double)w[c];
            if (tid == 0) wsum += w[c];
#pragma unroll
            for (int u = 0; u < kWlMaxQ; ++u) {
                const int q = tid + u * kWlThreads;
                if (q < d) acc[u] = __dadd_rn(acc[u], __dmul_rn(wc, (double)cand[(int64_t)c * d + q]));
            }
        }
        __syncthreads();
    }
    __shared__ long long s_w;
    if (tid == 0) s_w = wsum;
    __syncthreads();
    if (s_w == 0) return;
#pragma unroll
    for (int u = 0; u < kWlMaxQ; ++u) {
        const int q = tid + u * kWlThreads;
        if (q < d) centers[(int64_t)j * d + q] = (float)(acc[u] / (double)s_w);
    }
}

cudaError_t launch_weighted_centroids(const Ctx &c, int m, const int32_t *lab, float *centers) {
    if (c.d > kWlMaxQ * kWlThreads) return cudaErrorInvalidValue;
    weighted_centroid_kernel<<<c.k, kWlThreads, 0, c.stream>>>(c.C, c.w, lab, m, c.d, centers);
    count_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Lloyd: centroids
// A stable counting sort of the points by label (per-block histograms, a chunked
// column scan, one warp per block scattering in point order) puts every cluster's
// members in ascending point order; each cluster is then cut into fixed pieces of
// kPiece sorted members, one CTA sums a piece in FP64 (fixed order), and the
// pieces of a cluster are added in order.  The result does not depend on
// scheduling or on the GPU's SM count.
constexpr int kPiece = 256;

// per sort block b (sb points): hist[b][j] = #points with label j
__global__ void label_hist_kernel(const int32_t *__restrict__ labels, int64_t n, int k, int sb, int32_t *hist) {
    extern __shared__ int32_t h[];
    for (int j = threadIdx.x; j < k; j += blockDim.x) h[j] = 0;
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * sb;
    const int64_t b1 = min(n, b0 + sb);
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) atomicAdd(&h[labels[i]], 1);
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) hist[(int64_t)blockIdx.x * k + j] = h[j];
}

// column scan in two parallel passes over (32 columns) x (64-row chunks):
// chunk totals, then each chunk's offset = sum of the earlier chunks, rescanned
// row by row: hist[b][j] <- sum_{b' < b} hist[b'][j]; tot[j] = column total.
constexpr int kScanRows = 64;

__global__ void __launch_bounds__(256) column_chunk_kernel(const int32_t *__restrict__ hist, int nsb, int k,
                                                           int32_t *chunk) {
    __shared__ int part[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + lane, rc = blockIdx.y;
    const int b0 = rc * kScanRows + w * (kScanRows / 8);
    const int b1 = min(nsb, b0 + kScanRows / 8);
    int s = 0;
    if (j < k)
        for (int b = b0; b < b1; ++b) s += hist[(int64_t)b * k + j];
    part[w][lane] = s;
    __syncthreads();
    if (w == 0 && j < k) {
        int t = 0;
        for (int i = 0; i < 8; ++i) t += part[i][lane];
        chunk[(int64_t)rc * k + j] = t;
    }
}

__global__ void __launch_bounds__(256) column_offset_kernel(int32_t *hist, int nsb, int k,
                                                            const int32_t *__restrict__ chunk, int nrc, int32_t *tot) {
    __shared__ int part[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + lane, rc = blockIdx.y;
    // offset of this chunk (earlier chunks, split over the 8 warps, fixed order)
    int s = 0;
    if (j < k)
        for (int i = w; i < rc; i += 8) s += chunk[(int64_t)i * k + j];
    part[w][lane] = s;
    __syncthreads();
    int off = 0;
    for (int i = 0; i < 8; ++i) off += part[i][lane];
    if (rc == nrc - 1 && w == 0 && j < k) tot[j] = off + chunk[(int64_t)rc * k + j];
    __syncthreads();
    // per-warp prefix inside the chunk, then each warp rescans its rows
    const int b0 = rc * kScanRows + w * (kScanRows / 8);
    const int b1 = min(nsb, b0 + kScanRows / 8);
    int mine = 0;
    if (j < k)
        for (int b = b0; b < b1; ++b) mine += hist[(int64_t)b * k + j];
    part[w][lane] = mine;
    __syncthreads();
    int run = off;
    for (int i = 0; i < w; ++i) run += part[i][lane];
    if (j < k)
        for (int b = b0; b < b1; ++b) {
            const int64_t o = (int64_t)b * k + j;
            const int v = hist[o];
            hist[o] = run;
            run += v;
        }
}

// base[j] = sum_{j' < j} tot[j'] (base[k] = n) and piece[j] = sum_{j' < j}
// ceil(tot[j'] / kPiece) (piece[k] = number of pieces); one CTA, contiguous chunks
__global__ void __launch_bounds__(1024) base_scan_kernel(int32_t *tot_base, int k, int32_t *piece) {
    __shared__ int buf[1024], bufp[1024];
    const int t = threadIdx.x;
    const int q = (k + 1023) / 1024;
    const int lo = min(k, t * q), hi = min(k, lo + q);
    int local = 0, localp = 0;
    for (int j = lo; j < hi; ++j) {
        const int v = tot_base[j];
        local += v;
        localp += (v + kPiece - 1) / kPiece;
    }
    buf[t] = local;
    bufp[t] = localp;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int a = t >= off ? buf[t - off] : 0, ap = t >= off ? bufp[t - off] : 0;
        __syncthreads();
        buf[t] += a;
        bufp[t] += ap;
        __syncthreads();
    }
    int run = t > 0 ? buf[t - 1] : 0, runp = t > 0 ? bufp[t - 1] : 0;
    const int total = buf[1023], totalp = bufp[1023];
    __syncthreads();
    for (int j = lo; j < hi; ++j) {
        const int v = tot_base[j];
        tot_base[j] = run;
        piece[j] = runp;
        run += v;
        runp += (v + kPiece - 1) / kPiece;
    }
    if (t == 0) {
        tot_base[k] = total;
        piece[k] = totalp;
    }
}

// one warp per sort block: stable scatter of point numbers into label order
__global__ void __launch_bounds__(32) scatter_kernel(const int32_t *__restrict__ labels, int64_t n, int k, int sb,
                                                     const int32_t *__restrict__ hist,
                                                     const int32_t *__restrict__ base, int32_t *perm) {
    extern __shared__ int32_t cur[];
    const int lane = threadIdx.x;
    for (int j = lane; j < k; j += 32) cur[j] = base[j] + hist[(int64_t)blockIdx.x * k + j];
    __syncwarp();
    const int64_t b0 = (int64_t)blockIdx.x * sb;
    const int64_t b1 = min(n, b0 + sb);
    for (int64_t c0 = b0; c0 < b1; c0 += 32) {
        const int64_t i = c0 + lane;
        const bool valid = i < b1;
        const int l = valid ? labels[i] : -1;
        const unsigned mask = __match_any_sync(0xffffffffu, l);
        const int rank = __popc(mask & ((1u << lane) - 1u));
        if (valid) perm[cur[l] + rank] = (int32_t)i;
        __syncwarp();
        if (valid && lane == __ffs(mask) - 1) cur[l] += __popc(mask);
        __syncwarp();
    }
}

// Error-free accumulation of FP32 values: TwoSum (Knuth) keeps the exact rounding
// error of every addition; (s, c) carries at least 44 significant bits.  The
// rounded operations are explicit so that no reassociation can change them.
__device__ __forceinline__ void two_sum_add(float &s, float &c, float x) {
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    c = __fadd_rn(c, err);
    s = t;
}

// one CTA per piece: sum of up to kPiece sorted member rows.  Warp w takes members
// w, w + 8, ... in order with sixteen row loads in flight, lanes over coordinates:
// a lane carries a coordinate pair (8-byte loads, a whole 64-float slice of a row
// in one instruction) when rows are 8-byte aligned, else one coordinate; sums are
// compensated FP32 pairs (TwoSum), and the warps' sums are combined in FP64 in
// warp order.
constexpr int kPieceUnroll = 16;

// read-only loads kept in program order, so that a group of them is in flight
// together before the first one is used
__device__ __forceinline__ float2 ld_nc_f2(const float *p) {
    float2 v;
    asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
// an empty statement that takes eight values as in/out operands: the additions
// after it cannot move above it, so the loads before it are all issued first
__device__ __forceinline__ void hold8(float &a, float &b, float &c, float &d, float &e, float &f, float &g, float &h) {
    asm volatile("" : "+f"(a), "+f"(b), "+f"(c), "+f"(d), "+f"(e), "+f"(f), "+f"(g), "+f"(h));
}
__device__ __forceinline__ float ld_nc_f1(const float *p) {
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

__global__ void __launch_bounds__(256, 4) piece_sum_kernel(const float *__restrict__ X, int d, int k, int pairs,
                                                        const int32_t *__restrict__ perm,
                                                        const int32_t *__restrict__ base,
                                                        const int32_t *__restrict__ piece, double *psum) {
    __shared__ double part[8][64];
    __shared__ int rows[kPiece];
    __shared__ int s_j;
    const int pid = blockIdx.x;
    if (pid >= piece[k]) return;   // uniform per block
    if (threadIdx.x == 0) {
        int lo = 0, hi = k;        // the cluster whose piece range holds pid
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (piece[mid] <= pid) lo = mid; else hi = mid;
        }
        s_j = lo;
    }
    __syncthreads();
    const int j = s_j;
    const int p0 = base[j] + (pid - piece[j]) * kPiece;
    const int cnt = min(kPiece, base[j + 1] - p0);
    for (int i = threadIdx.x; i < cnt; i += 256) rows[i] = perm[p0 + i];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int per_pass = pairs ? 64 : 32;
    for (int dc = 0; dc < d; dc += per_pass) {
        float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
        if (pairs) {
            const int q = dc + 2 * lane;
            if (q < d) {
                int i = w;
                for (; i + 8 * (kPieceUnroll - 1) < cnt; i += 8 * kPieceUnroll) {
                    float2 v[kPieceUnroll];
#pragma unroll
                    for (int u = 0; u < kPieceUnroll; ++u) v[u] = ld_nc_f2(X + (int64_t)rows[i + 8 * u] * d + q);
#pragma unroll
                    for (int u = 0; u < kPieceUnroll; u += 4)
                        hold8(v[u].x, v[u].y, v[u + 1].x, v[u + 1].y, v[u + 2].x, v[u + 2].y, v[u + 3].x, v[u + 3].y);
#pragma unroll
                    for (int u = 0; u < kPieceUnroll; ++u) {
                        two_sum_add(sx, cx, v[u].x);
                        two_sum_add(sy, cy, v[u].y);
                    }
                }
                for (; i < cnt; i += 8) {
                    const float2 v = __ldg(reinterpret_cast<const float2 *>(X + (int64_t)rows[i] * d + q));
                    two_sum_add(sx, cx, v.x);
                    two_sum_add(sy, cy, v.y);
                }
            }
            part[w][2 * lane] = (double)sx + (double)cx;
            part[w][2 * lane + 1] = (double)sy + (double)cy;
        } else {
            const int q = dc + lane;
            if (q < d) {
                int i = w;
                for (; i + 8 * (kPieceUnroll - 1) < cnt; i += 8 * kPieceUnroll) {
                    float v[kPieceUnroll];
#pragma unroll
                    for (int u = 0; u < kPieceUnroll; ++u) v[u] = ld_nc_f1(X + (int64_t)rows[i + 8 * u] * d + q);
#pragma unroll
                    for (int u = 0; u < kPieceUnroll; u += 8)
                        hold8(v[u], v[u + 1], v[u + 2], v[u + 3], v[u + 4], v[u + 5], v[u + 6], v[u + 7]);
#pragma unroll
                    for (int u = 0; u < kPieceUnroll; ++u) two_sum_add(sx, cx, v[u]);
                }
                for (; i < cnt; i += 8) two_sum_add(sx, cx, __ldg(X + (int64_t)rows[i] * d + q));
            }
            part[w][lane] = (double)sx + (double)cx;
        }
        __syncthreads();
        if (w == 0) {
            for (int c = lane; c < per_pass && dc + c < d; c += 32) {
                double acc = 0.0;
                for (int u = 0; u < 8; ++u) acc += part[u][c];
                psum[(int64_t)pid * d + dc + c] = acc;
            }
        }
        __syncthreads();
    }
}

// per cluster: pieces added in order, centroid = sum / count rounded to FP32;
// an empty cluster keeps its center
__global__ void centroid_finalize_kernel(int d, int k, const int32_t *__restrict__ base,
                                         const int32_t *__restrict__ piece, const double *__restrict__ psum,
                                         float *centers) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)k * d) return;
    const int j = (int)(e / d), q = (int)(e - (int64_t)j * d);
    const int cnt = base[j + 1] - base[j];
    if (cnt == 0) return;
    double s = 0.0;
    for (int p = piece[j]; p < piece[j + 1]; ++p) s += psum[(int64_t)p * d + q];
    centers[e] = (float)__ddiv_rn(s, (double)cnt);
}

int sort_block_size(int64_t n, int k) {
    int sb = 512;
    while ((int64_t)((n + sb - 1) / sb) * k > (1ll << 26) && sb < (1 << 20)) sb <<= 1;
    return sb;
}

int64_t max_pieces(int64_t n, int k) { return (n + kPiece - 1) / kPiece + k; }

int64_t scan_chunks(int nsb) { return (nsb + kScanRows - 1) / kScanRows; }

cudaError_t launch_centroids(Ctx &c, const int32_t *labels, float *centers) {
    cudaError_t e;
    const int k = c.k, sb = c.sort_block;
    label_hist_kernel<<<c.nsb, 256, sizeof(int32_t) * k, c.stream>>>(labels, c.n, k, sb, c.hist);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int nrc = (c.nsb + kScanRows - 1) / kScanRows;
    column_chunk_kernel<<<dim3((k + 31) / 32, nrc), 256, 0, c.stream>>>(c.hist, c.nsb, k, c.chunk);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    column_offset_kernel<<<dim3((k + 31) / 32, nrc), 256, 0, c.stream>>>(c.hist, c.nsb, k, c.chunk, nrc, c.base);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    base_scan_kernel<<<1, 1024, 0, c.stream>>>(c.base, k, c.piece);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    scatter_kernel<<<c.nsb, 32, sizeof(int32_t) * k, c.stream>>>(labels, c.n, k, sb, c.hist, c.base, c.perm);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // coordinate pairs need 8-byte aligned rows: d even and X 8-byte aligned
    const int pairs = (c.d % 2 == 0) && (reinterpret_cast<uintptr_t>(c.X) % 8 == 0);
    piece_sum_kernel<<<(int)max_pieces(c.n, k), 256, 0, c.stream>>>(c.X, c.d, k, pairs, c.perm, c.base, c.piece,
                                                                    c.psum);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t kd = (int64_t)k * c.d;
    centroid_finalize_kernel<<<(int)((kd + 255) / 256), 256, 0, c.stream>>>(c.d, k, c.base, c.piece, c.psum, centers);
    count_launches(7);
    return cudaGetLastError();
}

}  // namespace kmp

namespace kmp {
cudaError_t configure_round_kernels(int max_sort_pow2);

cudaError_t configure_kernels(int max_sort_pow2, int k) {
    cudaError_t e = configure_round_kernels(max_sort_pow2);
    if (e != cudaSuccess) return e;
    const int hist_bytes = (int)sizeof(int32_t) * std::min(k, 49152);
    if (hist_bytes > 48 * 1024) {
        if ((e = cudaFuncSetAttribute(label_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, hist_bytes)) !=
            cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, hist_bytes)) !=
            cudaSuccess)
            return e;
    }
    return cudaSuccess;
}
}  // namespace kmp
