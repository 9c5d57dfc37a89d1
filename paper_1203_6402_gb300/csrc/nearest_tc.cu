// nearest_tc.cu -- the distance passes of k-means|| (Alg. 2 step 5, Sec. 3.3) and
// of Lloyd's assignment (Sec. 3.1) on the tcgen05 tensor cores of sm_103a.
//
// Screening: for a 128-row tile of X and a BN-column tile of centers, one
// tcgen05.mma chain (BF16 inputs, FP32 accumulator in TMEM) produces
//     s~(x, c) = ||c||^2 - 2 x.c        (= d^2(x, c) - ||x||^2)
// with ||c||^2 folded into two extra K columns (A row: [x..., 1, 1], B row:
// [-2c..., cn_hi, cn_lo]).  In split mode every coordinate is carried as hi + lo
// BF16 parts and three products (hi.hi, lo.hi, hi.lo) are summed, which brings the
// screening error from ~2^-6 to ~2^-13 of ||x|| ||c||.
//
// Epilogue (8 warps, one TMEM lane per row, two warps per lane quarter): each
// value becomes a key whose low 8 mantissa bits hold its column; a branch-free
// top-2 over the keys gives the best center and the runner-up value.  If the
// runner-up is outside the screening error window the best center is certain and
// is written out; the exact FP32 distance and the decision are then taken by
// refine_kernel exactly as on the CUDA-core path.  Otherwise the row goes to a
// fix-up list that the CUDA-core kernel finishes with an exact scan.  Decisions
// are therefore identical to the FP32 path.
//
// The A operand (points) is encoded once per context by prep_points_kernel into a
// swizzled BF16 image of X (one contiguous block per 128-row tile) together with
// ||x||^2; the B operand (centers) is encoded per pass by prep_centers_kernel.
//
// CTA roles (persistent, one CTA per SM, 320 threads):
//   warp 0      producer: bulk copies of A and B tiles into smem
//   warp 1      TMEM allocation, MMA issue (one lane)
//   warps 2-9   epilogue
// Every wait is bounded; on a timeout the kernel raises an error word, unwinds,
// waits (bounded) for its own copies and MMAs and frees its TMEM.
#include <cuda_bf16.h>
#include <float.h>

#include "kmpar_internal.cuh"
#include "nearest_tc.cuh"

namespace kmp {
namespace tc {

constexpr int kThreads = 320;
constexpr int BM = 128;
constexpr unsigned long long kWaitCycles = 4000000000ull;   // ~2 s at 2 GHz

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
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *holder, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(holder)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
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

// K-major operand, 128-byte swizzle: 8-row x 128 B atoms (1024 B), SBO = 1024 B.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}
// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, N = bn, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int bn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// byte offset of 16-byte chunk c of row r in a K-atom of an SW128 tile
__host__ __device__ __forceinline__ uint32_t sw128_off(int r, int c) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

// ------------------------------------------------------------------ operand encoding
struct Enc {
    int d;
    int split;   // 0: [x, 1, 1]; 1: [x_hi, x_lo, x_hi, 1, 1]
};

__device__ __forceinline__ __nv_bfloat16 bf(float v) { return __float2bfloat16_rn(v); }

// element k of the A (point) row
__device__ __forceinline__ __nv_bfloat16 a_elem(const Enc &e, const float *x, int k) {
    const int d = e.d;
    if (!e.split) {
        if (k < d) return bf(x[k]);
        if (k == d || k == d + 1) return bf(1.f);
        return bf(0.f);
    }
    if (k < d) return bf(x[k]);
    if (k < 2 * d) { const float v = x[k - d]; return bf(v - __bfloat162float(bf(v))); }
    if (k < 3 * d) return bf(x[k - 2 * d]);
    if (k == 3 * d || k == 3 * d + 1) return bf(1.f);
    return bf(0.f);
}

// element k of the B (center) row.  Pad rows (no center) get a huge FINITE squared
// norm, so their screened value stays finite: a key built from +inf would become
// a NaN once the column bits are or-ed into its mantissa.
__device__ __forceinline__ __nv_bfloat16 b_elem(const Enc &e, const float *c, float cn_hi, float cn_lo, bool pad, int k) {
    const int d = e.d;
    const int base = e.split ? 3 * d : d;
    if (pad) return k == base ? bf(1e30f) : bf(0.f);
    if (!e.split) {
        if (k < d) return bf(-2.f * c[k]);
        if (k == d) return bf(cn_hi);
        if (k == d + 1) return bf(cn_lo);
        return bf(0.f);
    }
    if (k < 2 * d) return bf(-2.f * c[k < d ? k : k - d]);
    if (k < 3 * d) { const float v = c[k - 2 * d]; return bf(-2.f * (v - __bfloat162float(bf(v)))); }
    if (k == 3 * d) return bf(cn_hi);
    if (k == 3 * d + 1) return bf(cn_lo);
    return bf(0.f);
}

__device__ __forceinline__ uint4 pack8(const __nv_bfloat16 (&v)[8]) {
    uint4 u;
    u.x = (uint32_t)__bfloat16_as_ushort(v[0]) | ((uint32_t)__bfloat16_as_ushort(v[1]) << 16);
    u.y = (uint32_t)__bfloat16_as_ushort(v[2]) | ((uint32_t)__bfloat16_as_ushort(v[3]) << 16);
    u.z = (uint32_t)__bfloat16_as_ushort(v[4]) | ((uint32_t)__bfloat16_as_ushort(v[5]) << 16);
    u.w = (uint32_t)__bfloat16_as_ushort(v[6]) | ((uint32_t)__bfloat16_as_ushort(v[7]) << 16);
    return u;
}

// ------------------------------------------------------------------ center tiles
// One thread per padded center row: squared norm (FP32, ascending), ||c||, the
// running max of ||c|| and the row's KA x 8 swizzled chunks of the B image
// [tile][katom][BN rows][128 B].
__global__ void prep_centers_kernel(const float *__restrict__ C, int d, int split, int KA, int BN, const DevState *st,
                                    int cnt_static, int round_mode, uint8_t *__restrict__ img, float *cnorm,
                                    unsigned int *cmax_bits) {
    const int begin = round_mode ? st->batch_begin : 0;
    const int cnt = round_mode ? st->batch_cnt : cnt_static;
    const int rows = ((cnt + BN - 1) / BN) * BN;
    const Enc e{d, split};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < rows; j += gridDim.x * blockDim.x) {
        const bool pad = j >= cnt;
        const float *c = C + (int64_t)(begin + (pad ? 0 : j)) * d;
        float cn = 0.f;
        if (!pad) {
            for (int q = 0; q < d; ++q) cn = __fmaf_rn(c[q], c[q], cn);
            const float nrm = sqrtf(cn);
            cnorm[j] = nrm;
            atomicMax(cmax_bits, __float_as_uint(nrm));
        }
        const float cn_hi = __bfloat162float(bf(cn));
        const float cn_lo = cn - cn_hi;
        const int t = j / BN, jj = j % BN;
        uint8_t *tile = img + (size_t)t * KA * BN * 128;
        for (int a = 0; a < KA; ++a) {
            for (int ch = 0; ch < 8; ++ch) {
                __nv_bfloat16 v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = b_elem(e, c, cn_hi, cn_lo, pad, a * 64 + ch * 8 + q);
                *reinterpret_cast<uint4 *>(tile + (size_t)a * BN * 128 + sw128_off(jj, ch)) = pack8(v);
            }
        }
    }
}

// One thread per (padded) point row: ||x||^2 (FP32, ascending) and the row's
// KA x 8 swizzled chunks of the A image [row tile][katom][128 rows][128 B].
__global__ void prep_points_kernel(const float *__restrict__ X, int64_t n, int64_t n_pad, int d, int split, int KA,
                                   uint8_t *__restrict__ img, float *__restrict__ xnorm) {
    const Enc e{d, split};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += (int64_t)gridDim.x * blockDim.x) {
        const bool valid = i < n;
        const float *x = X + (valid ? i : 0) * (int64_t)d;
        float xn = 0.f;
        if (valid)
            for (int q = 0; q < d; ++q) xn = __fmaf_rn(x[q], x[q], xn);
        xnorm[i] = xn;
        const int64_t t = i / BM;
        const int r = (int)(i % BM);
        uint8_t *tile = img + (size_t)t * KA * BM * 128;
        for (int a = 0; a < KA; ++a) {
            for (int ch = 0; ch < 8; ++ch) {
                __nv_bfloat16 v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = valid ? a_elem(e, x, a * 64 + ch * 8 + q) : bf(0.f);
                *reinterpret_cast<uint4 *>(tile + (size_t)a * BM * 128 + sw128_off(r, ch)) = pack8(v);
            }
        }
    }
}

// ------------------------------------------------------------------ the pass
struct Smem {
    uint64_t a_full[4], a_free[4];
    uint64_t b_full[8], b_empty[8];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t merge_full[2], merge_free[2];
    uint32_t tmem_base;
    int abort;
    float merge_k1[2][BM];
    float merge_k2[2][BM];
    int merge_t1[2][BM];
};

template <int KA, int BN>
struct Cfg {
    static constexpr int A16_BYTES = KA * BM * 128;
    static constexpr int B_BYTES = KA * BN * 128;
    static constexpr int HALF = BN / 2;
    static constexpr int CHUNKS = HALF / 32;
};

struct Bound {
    float ep, en;   // E(x, c) = ep ||x|| ||c|| + en (||x||^2 + ||c||^2)
};

__device__ __forceinline__ float err_bound(const Bound &b, float X, float c) {
    return b.ep * X * c + b.en * (X * X + c * c);
}

// bounded wait on an mbarrier phase; false if this or another warp gave up
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, volatile int *abort, int *err, int code) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = clock64();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort = 1;
            atomicCAS(err, 0, code);
            return false;
        }
        __nanosleep(64);
    }
}

// wait that ignores the abort flag (used to drain copies and MMAs before exit)
__device__ __forceinline__ void drain_bar(uint64_t *bar, uint32_t parity) {
    const unsigned long long t0 = clock64();
    while (!mbar_try(bar, parity) && clock64() - t0 < kWaitCycles) __nanosleep(64);
}

template <int KA, int BN, int S, int A16B, int MODE>
__global__ void __launch_bounds__(kThreads, 1) nearest_tc_kernel(TcParams p) {
    using C = Cfg<KA, BN>;
    extern __shared__ __align__(1024) uint8_t dsmem[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~(uintptr_t)1023);
    uint8_t *bst = base;                                   // S B stages
    uint8_t *a16 = bst + S * C::B_BYTES;                   // A16B A tiles
    Smem &sm = *reinterpret_cast<Smem *>(a16 + A16B * C::A16_BYTES);
    volatile int *abort = &sm.abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n = p.n;
    const int nrt = (int)((n + BM - 1) / BM);
    const int begin = (MODE == 1) ? p.st->batch_begin : 0;
    const int cnt = (MODE == 1) ? p.st->batch_cnt : p.cnt;
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
            mbar_init(&sm.acc_empty[i], 8);
            mbar_init(&sm.merge_full[i], 4);
            mbar_init(&sm.merge_free[i], 4);
        }
        for (int i = 0; i < S; ++i) {
            mbar_init(&sm.b_full[i], 1);
            mbar_init(&sm.b_empty[i], 1);
        }
        sm.abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(&sm.tmem_base, 2 * BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;

    if (cnt > 0 && warp == 0) {
        // ------------------------------------------------ producer (one lane)
        if (lane == 0) {
            int bt = 0, lt = 0;
            if (resident)
                for (int t = 0; t < T; ++t) {
                    mbar_expect_tx(&sm.b_full[t], C::B_BYTES);
                    bulk_g2s(bst + t * C::B_BYTES, p.bimg + (size_t)t * C::B_BYTES, C::B_BYTES, &sm.b_full[t]);
                }
            for (int rt = blockIdx.x; rt < nrt; rt += gridDim.x, ++lt) {
                const int ab = lt % A16B;
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
            const uint32_t idesc = idesc_bf16(BN);
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
                    const uint32_t a0 = su32(a16 + ab * C::A16_BYTES);
                    const uint32_t b0 = su32(bst + s * C::B_BYTES);
                    for (int ks = 0; ks < ksteps; ++ks) {
                        const int at = ks >> 2;
                        const uint32_t off = (uint32_t)(ks & 3) * 32u;
                        mma_bf16(tmem + (uint32_t)(buf * BN), sw128_desc(a0 + at * (BM * 128) + off),
                                 sw128_desc(b0 + at * (BN * 128) + off), idesc, ks > 0 ? 1u : 0u);
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
        // ------------------------------------------------ epilogue (warps 2-9)
        const int e = warp - 2;               // 0..7
        const int quarter = warp & 3;         // TMEM lane quarter this warp may read
        const int half = e >> 2;              // column half of each center tile
        const int row = quarter * 32 + lane;  // row within the tile
        const Bound bnd{p.ep, p.en};
        const float cmax = __uint_as_float(*p.cmax_bits);
        const float INF = __uint_as_float(0x7F800000u);
        int lt = 0, g = 0;
        for (int rt = blockIdx.x; rt < nrt; rt += gridDim.x, ++lt) {
            const int mb = lt & 1;
            float K1 = INF, K2 = INF;
            int T1 = 0;
            bool ok = true;
            for (int t = 0; t < T; ++t, ++g) {
                const int buf = g & 1;
                if (!wait_bar(&sm.acc_full[buf], (g >> 1) & 1, abort, p.err, 18)) { ok = false; break; }
                tc_fence_after();
                float k1 = INF, k2 = INF;
                const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * BN + half * C::HALF);
#pragma unroll
                for (int c = 0; c < C::CHUNKS; ++c) {
                    uint32_t r[32];
                    tmem_ld32(tbase + c * 32, r);
                    tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 32; q += 2) {
                        // key = value with its column in the low 8 mantissa bits
                        const uint32_t col = (uint32_t)(half * C::HALF + c * 32 + q);
                        const float a = __uint_as_float((r[q] & 0xFFFFFF00u) | col);
                        const float b = __uint_as_float((r[q + 1] & 0xFFFFFF00u) | (col + 1));
                        const float lo = fminf(a, b), hi = fmaxf(a, b);
                        k2 = min3f(fmaxf(k1, lo), k2, hi);
                        k1 = fminf(k1, lo);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.acc_empty[buf]);
                if (k1 < K1) { K2 = fminf(K1, k2); K1 = k1; T1 = t; }
                else K2 = min3f(K2, k1, k2);
            }
            if (!ok) break;
            // merge the two column halves through shared memory (bounded waits only)
            if (half == 1) {
                if (lt >= 2 && !wait_bar(&sm.merge_free[mb], ((lt - 2) >> 1) & 1, abort, p.err, 19)) break;
                sm.merge_k1[mb][row] = K1;
                sm.merge_k2[mb][row] = K2;
                sm.merge_t1[mb][row] = T1;
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.merge_full[mb]);
                continue;
            }
            if (!wait_bar(&sm.merge_full[mb], (lt >> 1) & 1, abort, p.err, 20)) break;
            {
                const float o1 = sm.merge_k1[mb][row], o2 = sm.merge_k2[mb][row];
                const int ot = sm.merge_t1[mb][row];
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.merge_free[mb]);
                const float m1v = __uint_as_float(__float_as_uint(o1) & 0xFFFFFF00u);
                const float k1v = __uint_as_float(__float_as_uint(K1) & 0xFFFFFF00u);
                if (m1v < k1v || (m1v == k1v && ot < T1)) { K2 = min3f(K1, o2, K2); K1 = o1; T1 = ot; }
                else K2 = min3f(K2, o1, o2);
            }
            // ---- certain winner -> refine_kernel; otherwise the row goes to the fix-up pass
            const int64_t R = (int64_t)rt * BM + row;
            if (R < n) {
                const int jl = T1 * BN + (int)(__float_as_uint(K1) & 0xFFu);
                const float v1 = __uint_as_float(__float_as_uint(K1) & 0xFFFFFF00u);
                const float v2 = __uint_as_float(__float_as_uint(K2) & 0xFFFFFF00u);
                bool single = false;
                if (jl < cnt) {
                    const float xn = fmaxf(p.xnorm[R], 0.f);
                    const float X = sqrtf(xn);
                    const float E1 = err_bound(bnd, X, p.cnorm[jl]);
                    const float slack1 = fabsf(v1) * 6.2e-5f + E1;   // + key truncation (2^-15 relative)
                    const float d1 = fmaxf(v1 + xn + slack1, 0.f);   // bound on the winner's d^2
                    const float ceff = fminf(cmax, X + sqrtf(d1));
                    const float Eo = err_bound(bnd, X, ceff);
                    const float W = fp32_tie_window(p.d);
                    // v2 lowered by its key truncation; stays +inf when there is no runner-up
                    const float v2lo = v2 >= 0.f ? v2 * (1.f - 6.2e-5f) : v2 * (1.f + 6.2e-5f);
                    single = (v2lo - Eo) > (v1 + slack1 + W * d1 + 1e-30f);
                }
                if (single) {
                    p.cand1[R] = begin + jl;
                } else {
                    p.cand1[R] = -1;
                    const int pos = atomicAdd(p.fix_cnt, 1);
                    p.fix_rows[pos] = (int32_t)R;
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * BN);
    }
}

// ------------------------------------------------------------------ host side
template <int KA, int BN, int S, int A16B>
static constexpr size_t smem_bytes() {
    return 1024 + (size_t)S * Cfg<KA, BN>::B_BYTES + (size_t)A16B * Cfg<KA, BN>::A16_BYTES + sizeof(Smem);
}

template <int KA, int BN, int S, int A16B, int MODE>
static cudaError_t launch_cfg(const TcParams &p, int grid, cudaStream_t s) {
    static_assert(smem_bytes<KA, BN, S, A16B>() <= 227 * 1024, "shared memory");
    static_assert(S <= 8 && A16B <= 4, "barrier arrays");
    constexpr size_t sm = smem_bytes<KA, BN, S, A16B>();
    auto kern = nearest_tc_kernel<KA, BN, S, A16B, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<grid, kThreads, sm, s>>>(p);
    count_launches(1);
    return cudaGetLastError();
}

// the configurations this library is built with; KA = K atoms of 64 BF16
template <int MODE>
static cudaError_t dispatch(const TcParams &p, int KA, int grid, cudaStream_t s) {
    if (KA == 1) return launch_cfg<1, 256, 4, 4, MODE>(p, grid, s);
    if (KA == 2) return launch_cfg<2, 256, 2, 2, MODE>(p, grid, s);
    if (KA == 3) return launch_cfg<3, 128, 2, 2, MODE>(p, grid, s);
    return cudaErrorInvalidValue;
}

int tc_katoms(int d, int split) {
    const int k = split ? 3 * d + 2 : d + 2;
    return (k + 63) / 64;
}

int tc_ksteps(int d, int split) {
    const int k = split ? 3 * d + 2 : d + 2;
    return (k + 15) / 16;
}

int tc_block_n(int d, int split) { return tc_katoms(d, split) <= 2 ? 256 : 128; }

bool tc_supported(int d, int split) { return d >= 1 && tc_katoms(d, split) <= 3; }

size_t tc_points_image_bytes(int d, int split, int64_t n) {
    const int64_t tiles = (n + BM - 1) / BM;
    return (size_t)tiles * tc_katoms(d, split) * BM * 128;
}

cudaError_t launch_prep_points(const float *X, int64_t n, int d, int split, uint8_t *img, float *xnorm,
                               cudaStream_t s) {
    const int64_t n_pad = ((n + BM - 1) / BM) * BM;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n_pad + 127) / 128, 8192));
    prep_points_kernel<<<grid, 128, 0, s>>>(X, n, n_pad, d, split, tc_katoms(d, split), img, xnorm);
    count_launches(1);
    return cudaGetLastError();
}

Bound make_bound(int d, int split) {
    // unit roundoff of BF16 round-to-nearest
    const double u = 1.0 / 256.0;
    const int K = tc_ksteps(d, split) * 16;
    const double acc = K * std::ldexp(1.0, -23);                 // FP32 accumulation, generous
    const double norm = u * u + (d + 2) * std::ldexp(1.0, -24);   // hi/lo split of ||c||^2 + its FP32 sum
    double ep = split ? 2.0 * (3.0 * u * u + 3.0 * u * u * u) : 2.0 * (2.0 * u + u * u);
    ep = 1.25 * (ep + 2.0 * acc * 1.1);
    const double en = 1.25 * (norm + acc);
    return Bound{(float)ep, (float)en};
}

cudaError_t launch_prep_centers(const float *C, int d, int split, const DevState *st, int cnt_static, int round_mode,
                                int cap_rows, uint8_t *img, float *cnorm, unsigned int *cmax_bits, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(cmax_bits, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const int KA = tc_katoms(d, split), BN = tc_block_n(d, split);
    const int rows = ((cap_rows + BN - 1) / BN) * BN;
    const int grid = std::max(1, std::min((rows + 127) / 128, 4096));
    prep_centers_kernel<<<grid, 128, 0, s>>>(C, d, split, KA, BN, st, cnt_static, round_mode, img, cnorm, cmax_bits);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_nearest_tc(TcParams p, int mode_round, int num_sms, cudaStream_t s) {
    const Bound b = make_bound(p.d, p.split);
    p.ep = b.ep;
    p.en = b.en;
    p.ksteps = tc_ksteps(p.d, p.split);
    const int KA = tc_katoms(p.d, p.split);
    const int rows = (int)((p.n + BM - 1) / BM);
    const int grid = std::max(1, std::min(rows, num_sms));
    return mode_round ? dispatch<1>(p, KA, grid, s) : dispatch<0>(p, KA, grid, s);
}

size_t tc_image_bytes(int d, int split, int cap_rows) {
    const int KA = tc_katoms(d, split), BN = tc_block_n(d, split);
    const int tiles = (cap_rows + BN - 1) / BN;
    return (size_t)tiles * KA * BN * 128;
}

}  // namespace tc
}  // namespace kmp
