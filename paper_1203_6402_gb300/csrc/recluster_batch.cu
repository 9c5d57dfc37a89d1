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
// Per snapshot, four launches on the context's stream and no wait between CTAs:
//   rs_update_kernel   D^2 of every candidate against the centers kept in the last
//                      snapshot (a sum stops once it reaches D^2: sums of
//                      non-negative terms never decrease), masses w D^2 as double
//                      floats, chunk (32) and block (256 candidates) totals;
//   rs_propose_kernel  one warp per proposal i: u from counter (p + i, 0, 0, 5),
//                      target u * total, then the block, the chunk and the candidate
//                      by prefix sums in ascending order;
//   rs_pair_kernel     squared distances between the proposals (lower triangle);
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
constexpr int kUpdThreads = 256;                   // candidates per update block (8 chunks)
constexpr int kChunksPerBlock = kUpdThreads / 32;
constexpr int kPropWarps = 4;                      // proposals per propose block
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

__device__ __forceinline__ double warp_incl_scan_f64_rs(double v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v = __dadd_rn(u, v);
    }
    return v;
}

// partial distances of candidate j (coordinates from the transposed copy) to G
// centers at once (rows of cs, stride d, the first nr valid), coordinates in
// ascending order, each center's sum t = y - c, s = fma(t, t, s); the candidate's
// coordinates are read once for the G centers.  Stops once every sum has reached
// lim (it can then no longer lower the minimum: sums of non-negative terms never
// decrease); s[g] = +inf for g >= nr.
template <int G, bool VEC>
__device__ __forceinline__ void group_dist2(const float *__restrict__ CT, int mp, int j, const float *cs, int nr,
                                            int d, float lim, float (&s)[G]) {
#pragma unroll
    for (int g = 0; g < G; ++g) s[g] = g < nr ? 0.f : __int_as_float(0x7f800000);
    int q = 0;
    for (; q + 16 <= d; q += 16) {
        float y[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) y[u] = __ldg(CT + (size_t)(q + u) * mp + j);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g < nr) {
                const float *c = cs + (size_t)g * d + q;
                if (VEC) {
#pragma unroll
                    for (int u = 0; u < 16; u += 4) {
                        const float4 c4 = *reinterpret_cast<const float4 *>(c + u);
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
                        const float t = __fsub_rn(y[u], c[u]);
                        s[g] = __fmaf_rn(t, t, s[g]);
                    }
                }
            }
        }
        bool done = true;
#pragma unroll
        for (int g = 0; g < G; ++g) done &= !(s[g] < lim);
        if (done) return;
    }
    for (; q < d; ++q) {
        const float y = __ldg(CT + (size_t)q * mp + j);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g < nr) {
                const float t = __fsub_rn(y, cs[(size_t)g * d + q]);
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

// D^2 against the centers kept in the last snapshot (FIRST: no D^2, mass w), the
// masses' chunk totals gch and block totals gblk (FP64 in ascending order).  The
// centers go through shared memory in groups of gcap rows; each thread takes its
// candidate against 8 of them per pass over its coordinates.
template <bool FIRST, bool VEC>
__global__ void __launch_bounds__(kUpdThreads) rs_update_kernel(const float *__restrict__ C,
                                                               const float *__restrict__ CT, int mp,
                                                               const long long *__restrict__ w,
                                                               const DevState *st, int d,
                                                               const int32_t *__restrict__ chosen,
                                                               const RsCtl *ctl, int gcap, float *__restrict__ D2,
                                                               double *__restrict__ gch, double *__restrict__ gblk) {
    extern __shared__ __align__(16) float csm[];
    __shared__ double s_ct[kChunksPerBlock];
    if (ctl->done) return;
    const int m = st->m;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int j = blockIdx.x * kUpdThreads + threadIdx.x;
    Df e = {0.f, 0.f};
    if (FIRST) {
        if (j < m) e = df_mass(weight_split(w[j]), 0.f, true);
    } else {
        const bool init = ctl->init != 0;
        const int a0 = init ? 0 : ctl->first_new, a1 = init ? 1 : ctl->t;
        float dj = __int_as_float(0x7f800000);
        if (j < m && !init) dj = D2[j];
        for (int ab = a0; ab < a1; ab += gcap) {
            const int na = min(gcap, a1 - ab);
            __syncthreads();   // the previous group's rows are no longer read
            for (int f = threadIdx.x; f < na * d; f += kUpdThreads) {
                const int a = f / d, q = f - a * d;
                csm[f] = C[(size_t)chosen[ab + a] * d + q];
            }
            __syncthreads();
            if (j < m) {
                for (int r0 = 0; r0 < na; r0 += 8) {
                    float s8[8];
                    group_dist2<8, VEC>(CT, mp, j, csm + (size_t)r0 * d, min(8, na - r0), d, dj, s8);
#pragma unroll
                    for (int g = 0; g < 8; ++g)
                        if (s8[g] < dj) dj = s8[g];
                }
            }
        }
        if (j < m) {
            D2[j] = dj;
            e = df_mass(weight_split(w[j]), dj, false);
        }
    }
    const Df incl = warp_incl_scan_df(e, lane);
    if (lane == 31) {
        const double tot = df_to_double(incl);
        gch[(size_t)blockIdx.x * kChunksPerBlock + wid] = tot;
        s_ct[wid] = tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int c = 0; c < kChunksPerBlock; ++c) b = __dadd_rn(b, s_ct[c]);
        gblk[blockIdx.x] = b;
    }
}

// one warp per proposal: the candidate whose prefix interval holds u * total
template <bool FIRST>
__global__ void __launch_bounds__(32 * kPropWarps) rs_propose_kernel(const long long *__restrict__ w,
                                                                    const float *__restrict__ D2,
                                                                    const DevState *st,
                                                                    const double *__restrict__ gch,
                                                                    const double *__restrict__ gblk, int nblk,
                                                                    RsCtl *ctl, uint64_t seed, int P,
                                                                    RsProp *__restrict__ props) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kPropWarps + (threadIdx.x >> 5);
    if (i >= P || ctl->done) return;
    const int m = st->m;
    // the total and each lane's range of blocks, in ascending order
    const int bpl = (nblk + 31) / 32;
    const int b0 = min(nblk, lane * bpl), b1 = min(nblk, b0 + bpl);
    double ls = 0.0;
    for (int b = b0; b < b1; ++b) ls = __dadd_rn(ls, gblk[b]);
    const double incl = warp_incl_scan_f64_rs(ls, lane);
    double excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0.0;
    const double total = __shfl_sync(0xffffffffu, incl, 31);
    if (!(total > 0.0)) {
        if (i == 0 && lane == 0) ctl->zero = 1;
        return;
    }
    const uint64_t ctr = FIRST ? 0ull : ctl->p + (uint64_t)i;
    const double u = uniform53(ctr, 0, FIRST ? TAG_RECLUSTER : TAG_RECLUSTER_RS, seed);
    const double target = __dmul_rn(u, total);
    int near = 0;
    // block: first lane whose inclusive prefix exceeds the target, then within its
    // range; if rounding leaves none, the last block with positive mass
    int blk = -1;
    double pre_b = 0.0;
    {
        const unsigned hit = __ballot_sync(0xffffffffu, incl > target);
        int L;
        if (hit) {
            L = __ffs(hit) - 1;
        } else {
            const unsigned pos = __ballot_sync(0xffffffffu, ls > 0.0);
            L = pos ? 31 - __clz(pos) : 0;
            near = 1;
        }
        if (lane == L) {
            double pre = excl;
            int lastp = -1;
            double pre_last = 0.0;
            for (int b = b0; b < b1; ++b) {
                const double g = gblk[b];
                const double nxt = __dadd_rn(pre, g);
                if (g > 0.0) { lastp = b; pre_last = pre; }
                if (nxt > target && blk < 0 && hit) { blk = b; pre_b = pre; }
                pre = nxt;
            }
            if (blk < 0) { blk = lastp; pre_b = pre_last; near = 1; }
        }
        blk = __shfl_sync(0xffffffffu, blk, L);
        pre_b = __shfl_sync(0xffffffffu, pre_b, L);
        near = __shfl_sync(0xffffffffu, near, L);
    }
    // chunk within the block (one lane, ascending), the same fallback
    int ch = -1;
    double pre_c = 0.0;
    if (lane == 0) {
        double pre = pre_b;
        int lastp = -1;
        double pre_last = 0.0;
        for (int c = 0; c < kChunksPerBlock; ++c) {
            const double g = gch[(size_t)blk * kChunksPerBlock + c];
            const double nxt = __dadd_rn(pre, g);
            if (g > 0.0) { lastp = c; pre_last = pre; }
            if (nxt > target && ch < 0) { ch = c; pre_c = pre; }
            pre = nxt;
        }
        if (ch < 0) { ch = lastp; pre_c = pre_last; near = 1; }
    }
    ch = __shfl_sync(0xffffffffu, ch, 0);
    pre_c = __shfl_sync(0xffffffffu, pre_c, 0);
    near = __shfl_sync(0xffffffffu, near, 0);
    // candidate within the chunk: the same masses as the update kernel's
    const int j = (blk * kChunksPerBlock + ch) * 32 + lane;
    Df e = {0.f, 0.f};
    if (j < m) e = df_mass(weight_split(w[j]), FIRST ? 0.f : D2[j], FIRST);
    const Df inclf = warp_incl_scan_df(e, lane);
    const double ev = df_to_double(e), ic = df_to_double(inclf);
    const double cum = __dadd_rn(pre_c, ic), cum0 = __dadd_rn(pre_c, __dsub_rn(ic, ev));
    const unsigned hit = __ballot_sync(0xffffffffu, j < m && cum > target);
    int pick;
    if (hit) {
        const int hl = __ffs(hit) - 1;
        pick = (blk * kChunksPerBlock + ch) * 32 + hl;
        const int nr = fabs(target - cum0) <= 1e-6 * total || fabs(cum - target) <= 1e-6 * total;
        near |= __shfl_sync(0xffffffffu, nr, hl);
    } else {
        const unsigned pos = __ballot_sync(0xffffffffu, j < m && ev > 0.0);
        pick = (blk * kChunksPerBlock + ch) * 32 + (pos ? 31 - __clz(pos) : 0);
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

// Dpp[i P + i'] = ||c_{j_i} - c_{j_i'}||^2 for i' < i, stopping at S_i
__global__ void __launch_bounds__(128) rs_pair_kernel(const float *__restrict__ C, int d, const RsProp *props,
                                                      int P, const RsCtl *ctl, float *__restrict__ Dpp) {
    if (ctl->done || ctl->zero) return;
    const int i = blockIdx.x;
    const RsProp pi = props[i];
    const float *a = C + (size_t)pi.j * d;
    for (int i2 = threadIdx.x; i2 < i; i2 += blockDim.x)
        Dpp[(size_t)i * P + i2] = dist2_rows_lim(a, C + (size_t)props[i2].j * d, d, pi.S);
}

// the proposals in order: kept iff v S_j < D(j); FIRST: proposal 0 is draw 0
template <bool FIRST>
__global__ void __launch_bounds__(kAcceptThreads) rs_accept_kernel(const RsProp *props, int P, int B,
                                                                  const float *__restrict__ Dpp, RsCtl *ctl,
                                                                  int32_t *__restrict__ chosen, DevState *st,
                                                                  int k) {
    // the proposals' v, then the P x P pair distances (lower triangle used), D(j),
    // S_j, j and near flags
    extern __shared__ double dsm[];
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
    double *sv = dsm;
    float *dpp = reinterpret_cast<float *>(sv + P);
    float *dcur = dpp + (size_t)P * P;
    float *sS = dcur + P;
    int *sj = reinterpret_cast<int *>(sS + P);
    int *snr = sj + P;
    for (int f = threadIdx.x; f < P * P; f += blockDim.x) {
        const int i = f / P, i2 = f - i * P;
        if (i2 < i) dpp[f] = Dpp[f];
    }
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const RsProp pr = props[i];
        sv[i] = pr.v;
        dcur[i] = pr.S;
        sS[i] = pr.S;
        sj[i] = pr.j;
        snr[i] = pr.near;
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const int t0 = ctl->t;
    int t = t0, pending = ctl->pending, nnear = 0;
    for (int i = 0; i < P && t < k && t - t0 < B; ++i) {
        int acc = 0, j = 0;
        if (lane == 0) {
            const double S = (double)sS[i], dj = (double)dcur[i];
            const double lhs = __dmul_rn(sv[i], S);
            pending |= snr[i];
            if (fabs(lhs - dj) <= 1e-4 * S) pending = 1;
            acc = lhs < dj;
            j = sj[i];
            if (acc) {
                chosen[t] = j;
                nnear += pending;
                pending = 0;
            }
        }
        acc = __shfl_sync(0xffffffffu, acc, 0);
        if (acc) {
            ++t;
            for (int i2 = i + 1 + lane; i2 < P; i2 += 32) dcur[i2] = fminf(dcur[i2], dpp[(size_t)i2 * P + i]);
            __syncwarp();
        }
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
    const int nblk = (c.cap_total + kUpdThreads - 1) / kUpdThreads;
    if ((size_t)nblk * (kChunksPerBlock + 1) > 2 * (size_t)((c.cap_total + 31) / 32) + 2048)
        return cudaErrorInvalidValue;
    if ((e = launch_transpose_cand(c)) != cudaSuccess) return e;
    RsCtl *ctl = reinterpret_cast<RsCtl *>(c.rs_buf);
    RsProp *props = reinterpret_cast<RsProp *>(reinterpret_cast<char *>(c.rs_buf) + 256);
    float *Dpp = reinterpret_cast<float *>(props + kRsMaxProposals);
    double *gch = c.rc_cmass;
    double *gblk = c.rc_cmass + (size_t)nblk * kChunksPerBlock;
    const size_t acc_smem = sizeof(double) * P + sizeof(float) * ((size_t)P * P + 2 * P) + sizeof(int) * 2 * P;
    // centers staged per update block: up to B rows, at most 96 KB
    const int gcap = std::max(1, std::min(B, 98304 / (4 * c.d)));
    const size_t upd_smem = sizeof(float) * (size_t)gcap * c.d;
    const bool vec = c.d % 4 == 0;
    auto upd = vec ? rs_update_kernel<false, true> : rs_update_kernel<false, false>;
    if (upd_smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(upd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)upd_smem)) != cudaSuccess)
        return e;
    if (acc_smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(rs_accept_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)acc_smem)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(ctl, 0, sizeof(RsCtl), c.stream)) != cudaSuccess) return e;
    const int pgrid = (P + kPropWarps - 1) / kPropWarps;
    // draw 0
    rs_update_kernel<true, false><<<nblk, kUpdThreads, 0, c.stream>>>(c.C, c.rCT, mp, c.w, c.st, c.d, c.chosen,
                                                                      ctl, gcap, c.rD2, gch, gblk);
    rs_propose_kernel<true><<<1, 32 * kPropWarps, 0, c.stream>>>(c.w, c.rD2, c.st, gch, gblk, nblk, ctl, c.seed,
                                                                 1, props);
    rs_accept_kernel<true><<<1, kAcceptThreads, 0, c.stream>>>(props, 1, 1, Dpp, ctl, c.chosen, c.st, c.k);
    count_launches(3);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // snapshots: at least ceil((k - 1) / B); more while the proposals of a
    // snapshot keep fewer than B (each snapshot keeps at least its first proposal)
    int need = (c.k - 1 + B - 1) / B, launched = 0;
    while (need > 0) {
        for (int s = 0; s < need; ++s) {
            upd<<<nblk, kUpdThreads, upd_smem, c.stream>>>(c.C, c.rCT, mp, c.w, c.st, c.d, c.chosen, ctl, gcap,
                                                           c.rD2, gch, gblk);
            rs_propose_kernel<false><<<pgrid, 32 * kPropWarps, 0, c.stream>>>(c.w, c.rD2, c.st, gch, gblk, nblk,
                                                                              ctl, c.seed, P, props);
            rs_pair_kernel<<<P, 128, 0, c.stream>>>(c.C, c.d, props, P, ctl, Dpp);
            rs_accept_kernel<false><<<1, kAcceptThreads, acc_smem, c.stream>>>(props, P, B, Dpp, ctl, c.chosen,
                                                                               c.st, c.k);
        }
        count_launches(4 * need);
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
