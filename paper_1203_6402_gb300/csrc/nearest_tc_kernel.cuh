// nearest_tc_kernel.cuh -- the tcgen05 screening pass of k-means|| (Alg. 2 step 5,
// Sec. 3.3) and of Lloyd's assignment (Sec. 3.1), as a template over the operand
// format and the epilogue.  Included by one translation unit per format.
//
// Screening: distances are translation invariant, so both operands are first
// moved by a fixed anchor a (the column means of X, computed once per context):
// x' = x - a, c' = c - a.  For a 128-row tile of X and a BN-column tile of
// centers one tcgen05.mma chain (FP32 accumulator in TMEM) produces the screened
// value
//     s~(x, c) = ||c'||^2 - 2 x'.c'        (= d^2(x, c) - ||x'||^2)
// either with ||c'||^2 folded into two extra K columns (BF16, BF16X3) or added by
// the epilogue with one FMA per value (BF16N, FP8: value = ||c'||^2 + f acc, with
// f = -2 s_x s_t, the product of the row's and the center tile's power-of-two
// scales, so the scaling is exact).
//
// Epilogue (16 warps, one TMEM lane per row, four warps per lane quarter, each on
// its own column group of every center tile):
//   EPI_PAIR  adjacent centers are taken in pairs; the value-only minimum of a
//             pair becomes a key whose low 6 mantissa bits hold the pair's number
//             within the group, and a branch-free top-2 over keys gives the best
//             pair and the smallest screened value outside it.  The refine kernel
//             computes the pair in exact FP32 and decides whether it is certain.
//   EPI_LIST  for rows the pair screening left undecided: every center whose
//             screened value is at most the row's threshold (computed from an
//             exact FP32 upper bound of the row's nearest distance plus twice the
//             screening bound) is listed, kListSlots per row and column group;
//             a 32-value chunk is tested by its minimum first, so rows only branch
//             on chunks that hold a listed center.
//
// CTA roles (persistent, one CTA per SM, 576 threads):
//   warp 0      producer: bulk copies of A and B tiles into smem
//   warp 1      TMEM allocation, MMA issue (one lane)
//   warps 2-17  epilogue
// Every wait is bounded; on a timeout the kernel raises an error word, unwinds,
// waits (bounded) for its own copies and MMAs and frees its TMEM.
#pragma once

#include <float.h>

#include "kmpar_internal.cuh"
#include "nearest_tc.cuh"

namespace kmp {
namespace tc {

constexpr int kEpiWarps = 16;                    // epilogue warps (4 per TMEM lane quarter)
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kThreads = 64 + kEpiThreads;       // + producer warp + MMA warp
constexpr int kGroups = kEpiWarps / 4;           // column groups per center tile
constexpr int kPrefetch = 3;                     // A tiles pulled into L2 ahead of the current one
constexpr int BM = 128;
constexpr unsigned long long kWaitCycles = 4000000000ull;   // ~2 s at 2 GHz
constexpr float kPadNorm = 1e30f;                // squared norm of a pad center: never a winner

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t su32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *holder, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(holder)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// D (TMEM, FP32) (+)= A B^T; BF16 x BF16
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
            dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
// D (TMEM, FP32) (+)= A B^T; e4m3 x e4m3
__device__ __forceinline__ void mma_e4m3(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(
            dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// the same wait, with the loaded registers as operands: no use of them can be
// scheduled before it
__device__ __forceinline__ void tmem_wait_ld_dep(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
          "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
          "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
          "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
        :: "memory");
}
// asynchronous global -> shared copies of 16 and 4 bytes (one commit group per call site)
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(su32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// K-major operand, 128-byte swizzle: 8-row x 128 B atoms (1024 B), SBO = 1024 B.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}
// instruction descriptors (M = 128, N = bn, both operands K-major, D = F32):
// kind::f16 with A = B = BF16 (type code 1); kind::f8f6f4 with A = B = E4M3 (type code 0)
__host__ __device__ constexpr uint32_t idesc_bf16(int bn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_e4m3(int bn) {
    return (1u << 4) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// mask of a key's value bits; the low kColBits mantissa bits carry a column
constexpr int kColBits = 6;
constexpr uint32_t kValMask = ~((1u << kColBits) - 1u);

// ------------------------------------------------------------------ the pass
struct Smem {
    uint64_t a_full[4], a_free[4];
    uint64_t b_full[8], b_empty[8];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t merge_full[2], merge_free[2];
    uint32_t tmem_base;
    int abort;
    int nrows;
    float merge_k1[2][kGroups - 1][BM];
    float merge_k2[2][kGroups - 1][BM];
    int merge_t1[2][kGroups - 1][BM];
};

template <int KA, int BN>
struct Cfg {
    static constexpr int A16_BYTES = KA * BM * 128;
    static constexpr int B_BYTES = KA * BN * 128;
    static constexpr int GW = BN / kGroups;   // columns per epilogue warp
    static constexpr int CHUNKS = GW / 32;
    static constexpr int NB = GW + 4;         // floats of one warp's norm buffer (+ the tile scale)
    static_assert(GW / 2 <= (1 << kColBits) && GW % 32 == 0, "pair field");
};

template <int KA, int BN, int S, int A16B, int EPI>
constexpr size_t smem_bytes() {
    return 1024 + (size_t)S * Cfg<KA, BN>::B_BYTES + (size_t)A16B * Cfg<KA, BN>::A16_BYTES + sizeof(Smem) +
           (EPI != EPI_PAIR ? sizeof(int32_t) * kListSlots * kEpiThreads : 0) +
           sizeof(float) * kEpiWarps * 2 * Cfg<KA, BN>::NB;
}

// bounded wait on an mbarrier phase; false if this or another warp gave up.  The
// first probes spin (the hand-offs between the producer, the MMA warp and the
// epilogue are on the critical path of every tile), later ones back off.
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, volatile int *abort, int *err, int code) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = clock64();
    for (int it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (*abort) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort = 1;
            atomicCAS(err, 0, code);
            return false;
        }
        if (it >= 256) __nanosleep(64);
    }
}

// wait that ignores the abort flag (used to drain copies and MMAs before exit)
__device__ __forceinline__ void drain_bar(uint64_t *bar, uint32_t parity) {
    const unsigned long long t0 = clock64();
    while (!mbar_try(bar, parity) && clock64() - t0 < kWaitCycles) __nanosleep(64);
}

// value of one accumulator column: as computed (norms in K columns), or
// ||c'||^2 + f acc (norms in the epilogue)
template <bool NE>
__device__ __forceinline__ float screened(uint32_t raw, float f, float nc) {
    return NE ? __fmaf_rn(__uint_as_float(raw), f, nc) : __uint_as_float(raw);
}
// two adjacent columns at once: with norms in the epilogue one packed FP32x2 FMA
// (each half rounded like the scalar FMA, so the values are the same)
template <bool NE>
__device__ __forceinline__ void screened2(uint32_t r0, uint32_t r1, float f, float n0, float n1, float &v0,
                                          float &v1) {
    if (!NE) {
        v0 = __uint_as_float(r0);
        v1 = __uint_as_float(r1);
        return;
    }
    uint64_t d;
    asm("{\n\t.reg .b64 ta, tb, tc;\n\tmov.b64 ta, {%1, %2};\n\tmov.b64 tb, {%3, %3};\n\tmov.b64 tc, {%4, %5};\n\t"
        "fma.rn.f32x2 %0, ta, tb, tc;\n\t}"
        : "=l"(d)
        : "r"(r0), "r"(r1), "r"(__float_as_uint(f)), "r"(__float_as_uint(n0)), "r"(__float_as_uint(n1)));
    v0 = __uint_as_float((uint32_t)d);
    v1 = __uint_as_float((uint32_t)(d >> 32));
}

// GS: centers per screened group (2: pairs; 4: groups of four adjacent centers,
// whose minimum costs fewer ALU operations per value; the refine then computes all
// four exactly)
template <int KA, int BN, int S, int A16B, int FMT, int EPI, int GS>
__global__ void __launch_bounds__(kThreads, 1) nearest_tc_kernel(TcParams p, int mode_round) {
    using C = Cfg<KA, BN>;
    constexpr bool NE = FMT == FMT_BF16N || FMT == FMT_FP8;
    constexpr bool PAIR = EPI != EPI_LIST;       // the best group and the best value outside it
    constexpr bool PLIST = EPI == EPI_PAIRLIST;  // and the listing of groups at or below thr
    static_assert(!PLIST || (GS == 4 && NE), "listing pair screening: groups of four, norms in the epilogue");
    extern __shared__ __align__(1024) uint8_t dsmem[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~(uintptr_t)1023);
    uint8_t *bst = base;                                   // S B stages
    uint8_t *a16 = bst + S * C::B_BYTES;                   // A16B A tiles
    Smem &sm = *reinterpret_cast<Smem *>(a16 + A16B * C::A16_BYTES);
    int32_t *lsm = reinterpret_cast<int32_t *>(&sm + 1);   // EPI_LIST: kListSlots x kEpiThreads
    // per epilogue warp, two buffers of its column group's norms (and the FP8 tile
    // scale), filled one tile ahead by cp.async
    float *nbuf = reinterpret_cast<float *>(lsm + (EPI != EPI_PAIR ? kListSlots * kEpiThreads : 0));
    volatile int *abort = &sm.abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int begin = mode_round ? p.st->batch_begin : 0;
    const int cnt = mode_round ? p.st->batch_cnt : p.cnt;
    const int T = (cnt + BN - 1) / BN;
    const bool resident = T <= S;
    const int ksteps = p.ksteps;

    if (threadIdx.x == 0) {
        for (int i = 0; i < A16B; ++i) {
            mbar_init(&sm.a_full[i], 1);
            mbar_init(&sm.a_free[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&sm.acc_full[i], 1);
            mbar_init(&sm.acc_empty[i], kEpiWarps);
            mbar_init(&sm.merge_full[i], 4 * (kGroups - 1));
            mbar_init(&sm.merge_free[i], 4);
        }
        for (int i = 0; i < S; ++i) {
            mbar_init(&sm.b_full[i], 1);
            mbar_init(&sm.b_empty[i], 1);
        }
        sm.abort = 0;
        sm.nrows = (EPI == EPI_LIST || p.nrows_dev) ? *p.nrows_dev : (int)p.n;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(&sm.tmem_base, 2 * BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    const int64_t n = sm.nrows;
    const int nrt = (int)((n + BM - 1) / BM);

    if (cnt > 0 && warp == 0) {
        // ------------------------------------------------ producer (one lane)
        if (lane == 0) {
            int bt = 0, lt = 0;
            if (resident)
                for (int t = 0; t < T; ++t) {
                    mbar_expect_tx(&sm.b_full[t], C::B_BYTES);
                    bulk_g2s(bst + t * C::B_BYTES, p.bimg + (size_t)t * C::B_BYTES, C::B_BYTES, &sm.b_full[t]);
                }
            // the A tiles of the next row tiles are pulled into L2 ahead of their copies
            for (int q = 1; q <= kPrefetch; ++q) {
                const int64_t rq = blockIdx.x + (int64_t)q * gridDim.x;
                if (rq < nrt) prefetch_l2(p.ximg + (size_t)rq * C::A16_BYTES, C::A16_BYTES);
            }
            for (int rt = blockIdx.x; rt < nrt; rt += gridDim.x, ++lt) {
                const int ab = lt % A16B;
                const int64_t rq = rt + (int64_t)(kPrefetch + 1) * gridDim.x;
                if (rq < nrt) prefetch_l2(p.ximg + (size_t)rq * C::A16_BYTES, C::A16_BYTES);
                if (lt >= A16B && !wait_bar(&sm.a_free[ab], ((lt - A16B) / A16B) & 1, abort, p.err, 11)) break;
                mbar_expect_tx(&sm.a_full[ab], C::A16_BYTES);
                bulk_g2s(a16 + ab * C::A16_BYTES, p.ximg + (size_t)rt * C::A16_BYTES, C::A16_BYTES, &sm.a_full[ab]);
                if (!resident) {
                    bool ok = true;
                    for (int t = 0; t < T; ++t, ++bt) {
                        const int s = bt % S;
                        if (!wait_bar(&sm.b_empty[s], ((bt / S) & 1) ^ 1, abort, p.err, 12)) { ok = false; break; }
                        mbar_expect_tx(&sm.b_full[s], C::B_BYTES);
                        bulk_g2s(bst + s * C::B_BYTES, p.bimg + (size_t)t * C::B_BYTES, C::B_BYTES, &sm.b_full[s]);
                    }
                    if (!ok) break;
                }
            }
            // drain every copy issued before the CTA exits
            for (int i = (lt > A16B ? lt - A16B : 0); i < lt; ++i) drain_bar(&sm.a_full[i % A16B], (i / A16B) & 1);
            if (resident)
                for (int t = 0; t < T; ++t) drain_bar(&sm.b_full[t], 0);
            else
                for (int i = (bt > S ? bt - S : 0); i < bt; ++i) drain_bar(&sm.b_full[i % S], (i / S) & 1);
        }
    } else if (cnt > 0 && warp == 1) {
        // ------------------------------------------------ MMA issuer (one lane)
        if (lane == 0) {
            const uint32_t idesc = FMT == FMT_FP8 ? idesc_e4m3(BN) : idesc_bf16(BN);
            int lt = 0, g = 0, bt = 0;
            for (int rt = blockIdx.x; rt < nrt; rt += gridDim.x, ++lt) {
                const int ab = lt % A16B;
                if (!wait_bar(&sm.a_full[ab], (lt / A16B) & 1, abort, p.err, 13)) break;
                tc_fence_after();
                bool ok = true;
                for (int t = 0; t < T; ++t, ++g) {
                    const int s = resident ? t : bt % S;
                    const uint32_t bpar = resident ? 0u : (uint32_t)((bt / S) & 1);
                    if (!wait_bar(&sm.b_full[s], bpar, abort, p.err, 14)) { ok = false; break; }
                    const int buf = g & 1;
                    if (!wait_bar(&sm.acc_empty[buf], ((g >> 1) & 1) ^ 1, abort, p.err, 15)) { ok = false; break; }
                    tc_fence_after();
                    // descriptors: the start-address field is (address >> 4) in the low
                    // bits, so each 32-byte K step adds a compile-time constant to the
                    // tile's base descriptor (this thread shares its SMSP with ALU-heavy
                    // epilogue warps: few ALU instructions per MMA keep the tensor pipe fed)
                    const uint64_t ad0 = sw128_desc(su32(a16 + ab * C::A16_BYTES));
                    const uint64_t bd0 = sw128_desc(su32(bst + s * C::B_BYTES));
                    const uint32_t dt = tmem + (uint32_t)(buf * BN);
#pragma unroll
                    for (int ks = 0; ks < KA * 4; ++ks) {
                        if (ks < ksteps) {
                            const uint64_t ao = (uint64_t)(((ks >> 2) * (BM * 128) + (ks & 3) * 32) >> 4);
                            const uint64_t bo = (uint64_t)(((ks >> 2) * (BN * 128) + (ks & 3) * 32) >> 4);
                            if (FMT == FMT_FP8) mma_e4m3(dt, ad0 + ao, bd0 + bo, idesc, ks > 0 ? 1u : 0u);
                            else mma_bf16(dt, ad0 + ao, bd0 + bo, idesc, ks > 0 ? 1u : 0u);
                        }
                    }
                    mma_commit(&sm.acc_full[buf]);
                    if (!resident) { mma_commit(&sm.b_empty[s]); ++bt; }
                }
                if (!ok) break;
                mma_commit(&sm.a_free[ab]);
            }
            // the last commit covers every MMA this thread issued
            if (g > 0) drain_bar(&sm.acc_full[(g - 1) & 1], ((g - 1) >> 1) & 1);
        }
    } else if (cnt > 0) {
        // ------------------------------------------------ epilogue (warps 2 .. 2+kEpiWarps-1)
        const int e = warp - 2;
        const int etid = threadIdx.x - 64;    // epilogue thread 0 .. kEpiThreads-1
        const int quarter = warp & 3;         // TMEM lane quarter this warp may read
        const int grp = e >> 2;               // column group of each center tile
        const int row = quarter * 32 + lane;  // row within the tile
        const float INF = __uint_as_float(0x7F800000u);
        // kValMask as a runtime value: held in a register, the column is then the
        // one immediate of a single logic op per key
        const uint32_t vmask = p.vmask;
        // norms of center tile tn into buffer slot: one 16-byte copy per lane (a
        // tile's copies were issued one tile earlier, so their latency is hidden)
        float *nbw = nbuf + (size_t)e * 2 * C::NB;
        auto prefetch_norms = [&](int tn, int slot) {
            if (NE) {
                float *dst = nbw + slot * C::NB;
                if (lane < C::GW / 4) cp_async16(dst + lane * 4, p.ncol + (size_t)tn * BN + grp * C::GW + lane * 4);
                if (FMT == FMT_FP8 && lane == C::GW / 4) cp_async4(dst + C::GW, p.tscale + tn);
                cp_async_commit();
            }
        };
        if (nrt > blockIdx.x) prefetch_norms(0, 0);
        int lt = 0, g = 0;
        for (int rt = blockIdx.x; rt < nrt; rt += gridDim.x, ++lt) {
            const int mb = lt & 1;
            const int64_t R = (int64_t)rt * BM + row;
            // per-row factor of the epilogue FMA: -2 s_x (s_t is applied per tile)
            float fx = -2.f;
            if (FMT == FMT_FP8) fx = R < n ? -2.f * p.xscale[R] : 0.f;
            // EPI_LIST: the row's threshold (pad rows list nothing)
            float thr = -INF;
            if (EPI != EPI_PAIR && R < n) thr = p.thr[R];
            // EPI_PAIRLIST: the same threshold for the groups' minimum keys (a key
            // differs from its value by less than 2^-17 relative: widened by 2^-16, a
            // group that holds a value <= thr always passes; its values are then tested
            // exactly); -inf once the list has overflowed
            float thrk = thr == -INF ? -INF : thr + fabsf(thr) * 1.52587890625e-5f;
            int lcount = 0;
            float K1 = INF, K2 = INF;
            int T1 = 0;
            bool ok = true;
            for (int t = 0; t < T; ++t, ++g) {
                const int buf = g & 1;
                const float *nct = nullptr;
                if (NE) {
                    // every lane is done with the other slot (tile g - 1): refill it with
                    // the next tile's norms, then wait for this tile's
                    __syncwarp();
                    prefetch_norms(t + 1 < T ? t + 1 : 0, (g + 1) & 1);
                    cp_async_wait<1>();
                    __syncwarp();
                    nct = nbw + (g & 1) * C::NB;
                }
                float f = fx;
                if (FMT == FMT_FP8) f = fx * nct[C::GW];
                if (!wait_bar(&sm.acc_full[buf], (g >> 1) & 1, abort, p.err, 18)) { ok = false; break; }
                tc_fence_after();
                // two independent top-2 chains (alternate column pairs), merged per tile
                float k1a = INF, k2a = INF, k1b = INF, k2b = INF;
                const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * BN + grp * C::GW);
                static_assert(C::CHUNKS <= 2, "one load round per tile");
#pragma unroll
                for (int c = 0; c < C::CHUNKS; c += 2) {
                    uint32_t r[2][32];
                    // the second chunk's load is in flight while the first chunk is
                    // reduced; once the warp's columns are all in registers the
                    // accumulator buffer goes back to the MMA warp, so the next tile's
                    // MMAs overlap this warp's remaining work
                    tmem_ld32(tbase + c * 32, r[0]);
                    tmem_wait_ld_dep(r[0]);
                    if (c + 1 < C::CHUNKS) {
                        tmem_ld32(tbase + (c + 1) * 32, r[1]);
                    } else {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&sm.acc_empty[buf]);
                    }
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {
                        if (c + cc >= C::CHUNKS) break;
                        if (cc == 1) {
                            tmem_wait_ld_dep(r[1]);
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&sm.acc_empty[buf]);
                        }
                        if (PAIR) {
#pragma unroll
                            for (int q = 0; q < 32; q += 8) {
                                // value-only minimum of each pair of adjacent centers, then a
                                // key: the pair minimum with the pair's number within the
                                // group in the low mantissa bits (a compile-time constant)
                                float nv[8];
                                if (NE) {
                                    const float4 n0 = *reinterpret_cast<const float4 *>(nct + (c + cc) * 32 + q);
                                    const float4 n1 = *reinterpret_cast<const float4 *>(nct + (c + cc) * 32 + q + 4);
                                    nv[0] = n0.x; nv[1] = n0.y; nv[2] = n0.z; nv[3] = n0.w;
                                    nv[4] = n1.x; nv[5] = n1.y; nv[6] = n1.z; nv[7] = n1.w;
                                } else {
#pragma unroll
                                    for (int u = 0; u < 8; ++u) nv[u] = 0.f;
                                }
                                float v[8];
#pragma unroll
                                for (int u = 0; u < 8; u += 2)
                                    screened2<NE>(r[cc][q + u], r[cc][q + u + 1], f, nv[u], nv[u + 1], v[u], v[u + 1]);
                                if (GS == 4) {
                                    // two groups of four: minimum, key, one top-2 insertion
                                    const uint32_t gc = (uint32_t)(((c + cc) * 32 + q) >> 2);
                                    const float m0 = fminf(min3f(v[0], v[1], v[2]), v[3]);
                                    const float m1 = fminf(min3f(v[4], v[5], v[6]), v[7]);
                                    const float a = __uint_as_float((__float_as_uint(m0) & vmask) | gc);
                                    const float b = __uint_as_float((__float_as_uint(m1) & vmask) | (gc + 1));
                                    const float lo = fminf(a, b), hi = fmaxf(a, b);
                                    if (PLIST && lo <= thrk) {
                                        // (rarely) list the centers at or below the row's threshold;
                                        // an overflowed list stops here (its row takes the list pass)
                                        const int col0 = t * BN + grp * C::GW + (c + cc) * 32 + q;
#pragma unroll
                                        for (int u = 0; u < 8; ++u) {
                                            if (v[u] <= thr) {
                                                if (lcount < kListSlots) lsm[lcount * kEpiThreads + etid] = col0 + u;
                                                ++lcount;
                                            }
                                        }
                                        if (lcount > kListSlots) thrk = -INF;
                                    }
                                    if ((q >> 3) & 1) {
                                        k2b = min3f(fmaxf(k1b, lo), k2b, hi);
                                        k1b = fminf(k1b, lo);
                                    } else {
                                        k2a = min3f(fmaxf(k1a, lo), k2a, hi);
                                        k1a = fminf(k1a, lo);
                                    }
                                    continue;
                                }
                                const uint32_t pc = (uint32_t)(((c + cc) * 32 + q) >> 1);
                                const float m0 = fminf(v[0], v[1]);
                                const float m1 = fminf(v[2], v[3]);
                                const float m2 = fminf(v[4], v[5]);
                                const float m3 = fminf(v[6], v[7]);
                                const float a = __uint_as_float((__float_as_uint(m0) & vmask) | pc);
                                const float b = __uint_as_float((__float_as_uint(m1) & vmask) | (pc + 1));
                                const float e2 = __uint_as_float((__float_as_uint(m2) & vmask) | (pc + 2));
                                const float f2 = __uint_as_float((__float_as_uint(m3) & vmask) | (pc + 3));
                                const float loa = fminf(a, b), hia = fmaxf(a, b);
                                const float lob = fminf(e2, f2), hib = fmaxf(e2, f2);
                                k2a = min3f(fmaxf(k1a, loa), k2a, hia);
                                k1a = fminf(k1a, loa);
                                k2b = min3f(fmaxf(k1b, lob), k2b, hib);
                                k1b = fminf(k1b, lob);
                            }
                        } else {
                            // EPI_LIST: the chunk's values, their minimum, and (rarely) the
                            // listing of the values at or below the threshold
                            float v[32];
#pragma unroll
                            for (int q = 0; q < 32; q += 4) {
                                float4 n4 = make_float4(0.f, 0.f, 0.f, 0.f);
                                if (NE) n4 = *reinterpret_cast<const float4 *>(nct + (c + cc) * 32 + q);
                                screened2<NE>(r[cc][q], r[cc][q + 1], f, n4.x, n4.y, v[q], v[q + 1]);
                                screened2<NE>(r[cc][q + 2], r[cc][q + 3], f, n4.z, n4.w, v[q + 2], v[q + 3]);
                            }
                            float m4[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                m4[u] = min3f(v[8 * u], v[8 * u + 1], v[8 * u + 2]);
                                m4[u] = min3f(m4[u], v[8 * u + 3], v[8 * u + 4]);
                                m4[u] = min3f(m4[u], v[8 * u + 5], v[8 * u + 6]);
                                m4[u] = fminf(m4[u], v[8 * u + 7]);
                            }
                            const float m = fminf(min3f(m4[0], m4[1], m4[2]), m4[3]);
                            if (m <= thr) {
                                const int col0 = t * BN + grp * C::GW + (c + cc) * 32;
#pragma unroll
                                for (int j = 0; j < 32; ++j) {
                                    if (v[j] <= thr) {
                                        if (lcount < kListSlots) lsm[lcount * kEpiThreads + etid] = col0 + j;
                                        ++lcount;
                                    }
                                }
                            }
                        }
                    }
                }
                if (PAIR) {
                    const float k1 = fminf(k1a, k1b);
                    const float k2 = min3f(fmaxf(k1a, k1b), k2a, k2b);
                    if (k1 < K1) { K2 = fminf(K1, k2); K1 = k1; T1 = t; }
                    else K2 = min3f(K2, k1, k2);
                }
            }
            if (!ok) break;
            if (EPI != EPI_PAIR) {
                // each column group writes its own part of the row's list
                if (R < n) {
                    p.lcnt[R * kGroups + grp] = lcount;
                    const int w = lcount < kListSlots ? lcount : kListSlots;
                    for (int s = 0; s < w; ++s) p.lst[(R * kGroups + grp) * kListSlots + s] = lsm[s * kEpiThreads + etid];
                }
                if (EPI == EPI_LIST) continue;
            }
            // merge the column groups through shared memory (bounded waits only)
            if (grp > 0) {
                if (lt >= 2 && !wait_bar(&sm.merge_free[mb], ((lt - 2) >> 1) & 1, abort, p.err, 19)) break;
                sm.merge_k1[mb][grp - 1][row] = K1;
                sm.merge_k2[mb][grp - 1][row] = K2;
                sm.merge_t1[mb][grp - 1][row] = T1;
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.merge_full[mb]);
                continue;
            }
            if (!wait_bar(&sm.merge_full[mb], (lt >> 1) & 1, abort, p.err, 20)) break;
            int J1;
            {
                float o1[kGroups - 1], o2[kGroups - 1];
                int ot[kGroups - 1];
#pragma unroll
                for (int q = 0; q < kGroups - 1; ++q) {
                    o1[q] = sm.merge_k1[mb][q][row];
                    o2[q] = sm.merge_k2[mb][q][row];
                    ot[q] = sm.merge_t1[mb][q][row];
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.merge_free[mb]);
                // (masked value, first center of the pair) order; equal masked values
                // of different pairs are near ties that the certainty test sends to
                // the fix-up anyway.  Group 0's columns start at 0 within the tile,
                // group q+1's at (q+1) GW; a key carries the pair number in the group.
                J1 = T1 * BN + GS * (int)(__float_as_uint(K1) & ~kValMask);
#pragma unroll
                for (int q = 0; q < kGroups - 1; ++q) {
                    const float m1v = __uint_as_float(__float_as_uint(o1[q]) & kValMask);
                    const float k1v = __uint_as_float(__float_as_uint(K1) & kValMask);
                    const int oj = ot[q] * BN + (q + 1) * C::GW + GS * (int)(__float_as_uint(o1[q]) & ~kValMask);
                    if (m1v < k1v || (m1v == k1v && oj < J1)) { K2 = min3f(K1, o2[q], K2); K1 = o1[q]; J1 = oj; }
                    else K2 = min3f(K2, o1[q], o2[q]);
                }
            }
            // ---- the best pair and the best screened value outside it; the refine
            // computes the pair exactly and decides whether it is certain
            if (R < n) {
                p.cand1[R] = J1 < cnt ? begin + J1 : -1;
                p.v2[R] = __uint_as_float(__float_as_uint(K2) & kValMask);
            }
        }
    }

    cp_async_wait<0>();   // norm copies still in flight (a no-op for the other roles)
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * BN);
    }
}

template <int KA, int BN, int S, int A16B, int FMT, int EPI, int GS>
cudaError_t launch_cfg(const TcParams &p, int mode_round, int grid, cudaStream_t s) {
    static_assert(smem_bytes<KA, BN, S, A16B, EPI>() <= 227 * 1024, "shared memory");
    static_assert(S <= 8 && A16B <= 4, "barrier arrays");
    constexpr size_t sm = smem_bytes<KA, BN, S, A16B, EPI>();
    auto kern = nearest_tc_kernel<KA, BN, S, A16B, FMT, EPI, GS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<grid, kThreads, sm, s>>>(p, mode_round);
    count_launches(1);
    return cudaGetLastError();
}

// the configurations of one format; KA = K atoms of 128 bytes
template <int FMT, int EPI, int GS = 2>
cudaError_t dispatch_fmt(const TcParams &p, int mode_round, int KA, int grid, cudaStream_t s) {
    if (KA == 1) return launch_cfg<1, 256, 4, 4, FMT, EPI, GS>(p, mode_round, grid, s);
    if (KA == 2) return launch_cfg<2, 256, 2, 2, FMT, EPI, GS>(p, mode_round, grid, s);
    if (KA == 3) return launch_cfg<3, 128, 2, 2, FMT, EPI, GS>(p, mode_round, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace tc
}  // namespace kmp
