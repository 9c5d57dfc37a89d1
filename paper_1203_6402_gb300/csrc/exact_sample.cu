// exact_sample.cu -- the exactly-l-per-round variant of Algorithm 2 step 4
// (Bahmani et al., Sec. 5.3, the runs of Fig. 5.1): L = floor(l) points per
// round without replacement, each successive draw proportional to D^2 among the
// points not drawn yet (D^2 as at the start of the round).
//
// Point x gets the exponential clock kappa_x = -ln(u_x) / D^2(x), u_x from
// counter (x, round, EXACT); the clocks ring in the order of successive
// D^2-proportional draws, so the sample is the L earliest clocks (equal clocks:
// lower x first).  Points with D^2 = 0 never ring; when fewer than L points have
// D^2 > 0, all of those are drawn.  Clocks are FP32: positive floats order like
// their bit patterns, so the L-th clock is found by a most-significant-digit
// radix select over the 32-bit keys (four 8-bit digits):
//   exact_keys_kernel    clocks, count of points with D^2 > 0, histogram of
//                        the top digit
//   exact_pick_kernel    one thread: the digit bin holding the remaining rank
//   exact_hist_kernel    histogram of the next digit among keys on the prefix
//   exact_select_kernel  keys below the L-th appended to the round's draws; keys
//                        equal to it listed apart; keys in the boundary window
//                        counted
//   exact_ties_kernel    one CTA: the needed ties, by ascending point
// The draws then go through sort_batch_kernel (ascending point order), as in
// every round.
#include <float.h>

#include <algorithm>

#include "kmpar_internal.cuh"

namespace kmp {

constexpr uint32_t TAG_EXACT = 4u;
constexpr int kTieCap = 1024;   // keys equal to the L-th one that can be ordered
constexpr uint32_t kNoClock = 0x7F800000u;   // +inf: D^2 = 0

struct ExactWork {
    unsigned int hist[256];
    unsigned int prefix;   // key bits fixed so far (the L-th key after the last digit)
    int rem;               // rank still to find among the keys on the prefix (1-based)
    int target;            // min(L, points with D^2 > 0)
    int npos;              // points with D^2 > 0
    int ntie;              // keys equal to the L-th one
    int win;               // keys within the boundary window of the L-th one
};

size_t exact_work_bytes() { return sizeof(ExactWork); }
int exact_tie_cap() { return kTieCap; }

// -ln(u) in FP32 with a few ulp of relative error: ln of u itself below 1/2, and
// of 1 - v with v = 1 - u (exact in FP64) above, so that clocks near zero keep
// their relative precision.  u = 0 gives +inf.
__device__ __forceinline__ float clock_exp(double u) {
    if (u < 0.5) return -logf((float)u);
    return -log1pf(-(float)(1.0 - u));
}

// warp-aggregated increment of a shared-memory histogram bin
__device__ __forceinline__ void hist_add(unsigned int *h, unsigned int bin, bool active) {
    const unsigned act = __ballot_sync(0xffffffffu, active);
    if (!active) return;
    const unsigned peers = __match_any_sync(act, bin);
    const int lane = threadIdx.x & 31;
    if (lane == __ffs(peers) - 1) atomicAdd(&h[bin], (unsigned int)__popc(peers));
}

__global__ void __launch_bounds__(256) exact_keys_kernel(const float *__restrict__ D2, int64_t n, uint32_t round,
                                                         uint64_t seed, uint32_t *keys, ExactWork *ws) {
    __shared__ unsigned int h[256];
    for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
    __syncthreads();
    int pos = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {   // uniform per warp
        const int64_t i = base + threadIdx.x;
        uint32_t bits = kNoClock;
        if (i < n) {
            const float dd = D2[i];
            if (dd > 0.f) {
                const float e = clock_exp(uniform53((uint64_t)i, round, TAG_EXACT, seed));
                bits = __float_as_uint(fminf(__fdiv_rn(e, dd), FLT_MAX));
                ++pos;
            }
            keys[i] = bits;
        }
        hist_add(h, bits >> 24, i < n);
    }
    for (int o = 16; o > 0; o >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, o);
    if ((threadIdx.x & 31) == 0 && pos) atomicAdd(&ws->npos, pos);
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (h[b]) atomicAdd(&ws->hist[b], h[b]);
}

// the digit at `shift` of the target-th smallest key: first bin whose cumulative
// count reaches the remaining rank; the histogram is cleared for the next digit
__global__ void exact_pick_kernel(ExactWork *ws, int L, int shift) {
    if (threadIdx.x != 0) return;
    if (shift == 24) {
        ws->target = min(L, ws->npos);
        ws->rem = ws->target;
        ws->prefix = 0;
    }
    if (ws->target > 0) {
        unsigned int cum = 0;
        int b = 0;
        for (; b < 255; ++b) {
            if (cum + ws->hist[b] >= (unsigned int)ws->rem) break;
            cum += ws->hist[b];
        }
        ws->rem -= (int)cum;
        ws->prefix |= (unsigned int)b << shift;
    }
    for (int j = 0; j < 256; ++j) ws->hist[j] = 0;
}

__global__ void __launch_bounds__(256) exact_hist_kernel(const uint32_t *__restrict__ keys, int64_t n, ExactWork *ws,
                                                         int shift) {
    if (ws->target == 0) return;   // uniform: nothing to draw
    __shared__ unsigned int h[256];
    for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const uint32_t hi_mask = ~0u << (shift + 8);
    const uint32_t want = ws->prefix & hi_mask;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        const uint32_t bits = i < n ? keys[i] : 0u;
        const bool on = i < n && (bits & hi_mask) == want;
        hist_add(h, (bits >> shift) & 255u, on);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (h[b]) atomicAdd(&ws->hist[b], h[b]);
}

__global__ void __launch_bounds__(256) exact_select_kernel(const uint32_t *__restrict__ keys, int64_t n,
                                                           ExactWork *ws, DevState *st, int32_t *drawn, int cap,
                                                           int32_t *ties, float w) {
    if (ws->target == 0) return;
    const uint32_t T = ws->prefix;
    const float Tf = __uint_as_float(T);
    const float lo = Tf - w * Tf, hi = Tf + w * Tf;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {   // uniform per warp
        const int64_t i = base + threadIdx.x;
        const uint32_t bits = i < n ? keys[i] : kNoClock;
        const bool take = bits < T;
        const unsigned mask = __ballot_sync(0xffffffffu, take);
        if (mask) {
            const int leader = __ffs(mask) - 1;
            int b = 0;
            if (lane == leader) b = atomicAdd(&st->drawn, __popc(mask));
            b = __shfl_sync(0xffffffffu, b, leader);
            if (take) {
                const int p = b + __popc(mask & ((1u << lane) - 1u));
                if (p < cap) drawn[p] = (int32_t)i;
                else st->overflow = 1;
            }
        }
        if (bits == T) {
            const int p = atomicAdd(&ws->ntie, 1);
            if (p < kTieCap) ties[p] = (int32_t)i;
        }
        if (bits != kNoClock) {
            const float kf = __uint_as_float(bits);
            if (kf >= lo && kf <= hi) atomicAdd(&ws->win, 1);
        }
    }
}

// one CTA: the ties at the L-th key in ascending point order; the first rem of
// them complete the round's draws
__global__ void __launch_bounds__(1024) exact_ties_kernel(ExactWork *ws, DevState *st, const int32_t *ties,
                                                          int32_t *drawn, int cap, int L) {
    __shared__ int32_t s[kTieCap];
    __shared__ int base;
    if (ws->target == 0) return;   // uniform
    const int nt = min(ws->ntie, kTieCap);
    int P = 1;
    while (P < nt) P <<= 1;
    for (int e = threadIdx.x; e < P; e += blockDim.x) s[e] = e < nt ? ties[e] : INT_MAX;
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int e = threadIdx.x; e < P; e += blockDim.x) {
                const int o = e ^ stride;
                if (o > e) {
                    const bool asc = (e & size) == 0;
                    const int a = s[e], b = s[o];
                    if ((a > b) == asc) { s[e] = b; s[o] = a; }
                }
            }
        }
    }
    if (threadIdx.x == 0) base = st->drawn;
    __syncthreads();
    const int rem = min(ws->rem, nt);
    for (int j = threadIdx.x; j < rem; j += blockDim.x) {
        const int p = base + j;
        if (p < cap) drawn[p] = s[j];
    }
    if (threadIdx.x == 0) {
        st->drawn = base + rem;
        if (base + rem > cap || ws->ntie > kTieCap || ws->rem > nt) st->overflow = 1;
        if (ws->npos > L && ws->win >= 2) atomicAdd(&st->sample_near, 1ull);
    }
}

cudaError_t launch_sample_exact(Ctx &c, int round) {
    cudaError_t e;
    const int L = (int)std::min<double>(floor(c.ell), (double)c.cap_round);
    // window in which another clock may swap places with the L-th one between FP32
    // and exact arithmetic: D^2 carries (d + 1) 2^-24, the clock a few ulp more
    const float w = (float)((2.0 * c.d + 16.0) * 5.9604644775390625e-8);
    const int grid = c.num_sms * 8;
    ExactWork *ws = static_cast<ExactWork *>(c.ex_ws);
    if ((e = cudaMemsetAsync(ws, 0, sizeof(ExactWork), c.stream)) != cudaSuccess) return e;
    exact_keys_kernel<<<grid, 256, 0, c.stream>>>(c.D2, c.n, (uint32_t)round, c.seed, c.ex_keys, ws);
    exact_pick_kernel<<<1, 32, 0, c.stream>>>(ws, L, 24);
    for (int shift = 16; shift >= 0; shift -= 8) {
        exact_hist_kernel<<<grid, 256, 0, c.stream>>>(c.ex_keys, c.n, ws, shift);
        exact_pick_kernel<<<1, 32, 0, c.stream>>>(ws, L, shift);
    }
    exact_select_kernel<<<grid, 256, 0, c.stream>>>(c.ex_keys, c.n, ws, c.st, c.drawn, c.cap_round, c.ex_ties, w);
    exact_ties_kernel<<<1, 1024, 0, c.stream>>>(ws, c.st, c.ex_ties, c.drawn, c.cap_round, L);
    count_launches(10);
    return cudaGetLastError();
}

}  // namespace kmp
