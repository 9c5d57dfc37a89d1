// nearest_tc.cu -- the distance passes of k-means|| (Alg. 2 step 5, Sec. 3.3) and
// of Lloyd's assignment (Sec. 3.1) on the tcgen05 tensor cores of sm_103a.
//
// Screening: distances are translation invariant, so both operands are first
// moved by a fixed anchor a (the column means of X, computed once per context):
// x' = x - a, c' = c - a.  For a 128-row tile of X and a BN-column tile of
// centers, one tcgen05.mma chain (BF16 inputs, FP32 accumulator in TMEM) produces
//     s~(x, c) = ||c'||^2 - 2 x'.c'        (= d^2(x, c) - ||x'||^2)
// with ||c'||^2 folded into two extra K columns (A row: [x'..., 1, 1], B row:
// [-2c'..., cn_hi, cn_lo]).  In split mode every coordinate is carried as hi + lo
// BF16 parts and three products (hi.hi, lo.hi, hi.lo) are summed, which brings the
// screening error from ~2^-6 to ~2^-13 of ||x'|| ||c'||; the anchor makes those
// norms, and so the error, smaller for data away from the origin.
//
// Epilogue (16 warps, one TMEM lane per row, four warps per lane quarter, each on
// its own column group): adjacent centers are taken in pairs; the value-only
// minimum of a pair becomes a key whose low 6 mantissa bits hold the pair's number
// within the group (a compile-time constant: one logic op per pair), and a
// branch-free top-2 over the keys gives the best pair and the smallest screened
// value outside it (about 2.25 ALU ops per value, against 3.5 for a top-2 over
// single centers).  The refine kernel then computes both centers of the pair in
// exact FP32 and tests the other pairs' screened minimum against the error
// window: a certain row takes the CUDA-core decision on the pair; otherwise it
// goes to a fix-up list finished by an exact scan.  Decisions are therefore
// identical to the FP32 path.
//
// The A operand (points) is encoded once per context by prep_points_kernel into a
// swizzled BF16 image of X (one contiguous block per 128-row tile) together with
// ||x||^2; the B operand (centers) is encoded per pass by prep_centers_kernel.
//
// CTA roles (persistent, one CTA per SM, 576 threads):
//   warp 0      producer: bulk copies of A and B tiles into smem
//   warp 1      TMEM allocation, MMA issue (one lane)
//   warps 2-17  epilogue
// Every wait is bounded; on a timeout the kernel raises an error word, unwinds,
// waits (bounded) for its own copies and MMAs and frees its TMEM.
#include <cuda_bf16.h>
#include <float.h>

#include "kmpar_internal.cuh"
#include "nearest_tc.cuh"

namespace kmp {
namespace tc {

constexpr int kEpiWarps = 16;                    // epilogue warps (4 per TMEM lane quarter)
constexpr int kThreads = 64 + 32 * kEpiWarps;   // + producer warp + MMA warp
constexpr int kGroups = kEpiWarps / 4;          // column groups per center tile
constexpr int kPrefetch = 3;                    // A tiles pulled into L2 ahead of the current one
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
    int split;        // 0: [x', 1, 1]; 1: [x'_hi, x'_lo, x'_hi, 1, 1]
    const float *a;   // anchor: x' = fl(x - a), c' = fl(c - a)
};

// mask of a key's value bits; the low kColBits mantissa bits carry a column
constexpr int kColBits = 6;
constexpr uint32_t kValMask = ~((1u << kColBits) - 1u);

__device__ __forceinline__ __nv_bfloat16 bf(float v) { return __float2bfloat16_rn(v); }

// element k of the A (point) row
// x'_q = fl(x_q - a_q); a row already moved (e.a == nullptr) is used as it is
__device__ __forceinline__ float moved(const Enc &e, const float *x, int q) {
    return e.a ? __fsub_rn(x[q], e.a[q]) : x[q];
}

__device__ __forceinline__ __nv_bfloat16 a_elem(const Enc &e, const float *x, int k) {
    const int d = e.d;
    if (!e.split) {
        if (k < d) return bf(moved(e, x, k));
        if (k == d || k == d + 1) return bf(1.f);
        return bf(0.f);
    }
    if (k < d) return bf(moved(e, x, k));
    if (k < 2 * d) { const float v = moved(e, x, k - d); return bf(v - __bfloat162float(bf(v))); }
    if (k < 3 * d) return bf(moved(e, x, k - 2 * d));
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
        if (k < d) return bf(-2.f * moved(e, c, k));
        if (k == d) return bf(cn_hi);
        if (k == d + 1) return bf(cn_lo);
        return bf(0.f);
    }
    if (k < 2 * d) return bf(-2.f * moved(e, c, k < d ? k : k - d));
    if (k < 3 * d) { const float v = moved(e, c, k - 2 * d); return bf(-2.f * (v - __bfloat162float(bf(v)))); }
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
// One warp per padded center row: the moved row c' = fl(c - anchor) is staged in
// shared memory, lane 0 sums ||c'||^2 (FP32, ascending) and records the running max
// of ||c'||, and lanes 0 .. 8 KA - 1 build the row's 16-byte chunks of the B image
// [tile][katom][BN rows][128 B] in parallel.
constexpr int kPrepMaxD = 192;

__global__ void __launch_bounds__(256) prep_centers_kernel(const float *__restrict__ C, int d, int split, int KA, int BN,
                                                           const DevState *st, int cnt_static, int round_mode,
                                                           const float *__restrict__ anchor, uint8_t *__restrict__ img,
                                                           unsigned int *cmax_bits) {
    __shared__ float crow[8][kPrepMaxD];
    const int begin = round_mode ? st->batch_begin : 0;
    const int cnt = round_mode ? st->batch_cnt : cnt_static;
    const int rows = ((cnt + BN - 1) / BN) * BN;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const Enc em{d, split, nullptr};   // the staged row is already moved
    float *cr = crow[w];
    for (int j = blockIdx.x * 8 + w; j < rows; j += gridDim.x * 8) {   // uniform per warp
        const bool pad = j >= cnt;
        const float *c = C + (int64_t)(begin + (pad ? 0 : j)) * d;
        if (!pad)
            for (int q = lane; q < d; q += 32) cr[q] = __fsub_rn(c[q], anchor[q]);
        __syncwarp();
        float cn = 0.f;
        if (!pad && lane == 0) {
            for (int q = 0; q < d; ++q) cn = __fmaf_rn(cr[q], cr[q], cn);
            atomicMax(cmax_bits, __float_as_uint(sqrtf(cn)));
        }
        cn = __shfl_sync(0xffffffffu, cn, 0);
        const float cn_hi = __bfloat162float(bf(cn));
        const float cn_lo = cn - cn_hi;
        if (lane < KA * 8) {
            const int a = lane >> 3, ch = lane & 7;
            const int t = j / BN, jj = j % BN;
            uint8_t *tile = img + (size_t)t * KA * BN * 128;
            __nv_bfloat16 v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = b_elem(em, cr, cn_hi, cn_lo, pad, a * 64 + ch * 8 + q);
            *reinterpret_cast<uint4 *>(tile + (size_t)a * BN * 128 + sw128_off(jj, ch)) = pack8(v);
        }
        __syncwarp();   // the staged row is read before the next one overwrites it
    }
}

// One CTA per 128-row tile of the A image [row tile][katom][128 rows][128 B]: the
// tile's rows (contiguous in X) come into shared memory with coalesced loads; then
// eight consecutive threads build the eight 16-byte chunks of one row segment of an
// atom (position p of row r holds logical chunk p ^ (r & 7)), so the stores are
// coalesced too; thread r sums ||x'||^2 of row r (FP32, ascending; x' = x - anchor).
__global__ void __launch_bounds__(128) prep_points_kernel(const float *__restrict__ X, int64_t n, int64_t n_pad, int d,
                                                          int split, int KA, const float *__restrict__ anchor,
                                                          uint8_t *__restrict__ img, float *__restrict__ xnorm) {
    extern __shared__ float xsm[];   // BM x d
    const Enc e{d, split, anchor};
    const int64_t ntile = n_pad / BM;
    for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int64_t r0 = t * BM;
        const int nr = (int)max((int64_t)0, min((int64_t)BM, n - r0));
        __syncthreads();   // the previous tile's readers are done
        for (int f = threadIdx.x; f < nr * d; f += BM) xsm[f] = __ldg(X + r0 * d + f);
        __syncthreads();
        {
            const int r = threadIdx.x;
            float xn = 0.f;
            if (r < nr)
                for (int q = 0; q < d; ++q) {
                    const float v = moved(e, xsm + r * d, q);
                    xn = __fmaf_rn(v, v, xn);
                }
            xnorm[r0 + r] = xn;
        }
        uint8_t *tile = img + (size_t)t * KA * BM * 128;
        const int pos = threadIdx.x & 7;
        for (int a = 0; a < KA; ++a)
            for (int r = threadIdx.x >> 3; r < BM; r += BM / 8) {
                const int ch = pos ^ (r & 7);
                __nv_bfloat16 v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = r < nr ? a_elem(e, xsm + r * d, a * 64 + ch * 8 + q) : bf(0.f);
                *reinterpret_cast<uint4 *>(tile + (size_t)a * BM * 128 + r * 128 + pos * 16) = pack8(v);
            }
    }
}

// ------------------------------------------------------------------ anchor
// Column means of X, the anchor both operands are moved by.  Any anchor gives the
// same decisions (distances do not depend on it); the mean keeps ||x'|| small.
// kAnchorBlocks fixed row chunks; in a block, thread (ty, tx) sums column
// cc + tx over the chunk's rows ty, ty + 4, ... (warps read 32 consecutive
// floats of a row) in four FP32 chains of at most ~31 rows each (FP64 adds run
// at a small fraction of the FP32 rate here, and the anchor needs no more than
// FP32 accuracy); the chains, the four row phases, then the chunks, are added in
// FP64 in a fixed order, so the result is deterministic.
constexpr int kAnchorBlocks = 1024;

__global__ void __launch_bounds__(256) anchor_partial_kernel(const float *__restrict__ X, int64_t n, int d,
                                                             double *__restrict__ part) {
    __shared__ double ph[4][64];
    const int64_t chunk = (n + kAnchorBlocks - 1) / kAnchorBlocks;
    const int64_t r0 = (int64_t)blockIdx.x * chunk;
    const int64_t r1 = min(n, r0 + chunk);
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    for (int cc = 0; cc < d; cc += 64) {
        const int q = cc + tx;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        if (q < d) {
            int64_t r = r0 + ty;
            for (; r + 12 < r1; r += 16) {
                s0 += __ldg(X + r * d + q);
                s1 += __ldg(X + (r + 4) * d + q);
                s2 += __ldg(X + (r + 8) * d + q);
                s3 += __ldg(X + (r + 12) * d + q);
            }
            for (; r < r1; r += 4) s0 += __ldg(X + r * d + q);
        }
        ph[ty][tx] = (((double)s0 + (double)s1) + (double)s2) + (double)s3;
        __syncthreads();
        if (ty == 0 && q < d) part[(size_t)blockIdx.x * d + q] = ((ph[0][tx] + ph[1][tx]) + ph[2][tx]) + ph[3][tx];
        __syncthreads();
    }
}

// one block per column: thread t adds chunks t, t + 256, ... in order, then a fixed
// pairwise tree over the 256 partial sums
__global__ void __launch_bounds__(256) anchor_final_kernel(const double *__restrict__ part, int64_t n, int d,
                                                           float *__restrict__ anchor) {
    __shared__ double red[256];
    const int q = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < kAnchorBlocks; b += 256) s += part[(size_t)b * d + q];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) anchor[q] = n > 0 ? (float)(red[0] / (double)n) : 0.f;
}

// ------------------------------------------------------------------ the pass
struct Smem {
    uint64_t a_full[4], a_free[4];
    uint64_t b_full[8], b_empty[8];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t merge_full[2], merge_free[2];
    uint32_t tmem_base;
    int abort;
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
    static_assert(GW / 2 <= (1 << kColBits) && GW % 32 == 0, "pair field");
};

struct Bound {
    float ep, en;   // E(x, c) = ep ||x|| ||c|| + en (||x||^2 + ||c||^2)
};

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
            mbar_init(&sm.acc_empty[i], kEpiWarps);
            mbar_init(&sm.merge_full[i], 4 * (kGroups - 1));
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
                    // descriptors: the start-address field is (address >> 4) in the low
                    // bits, so each K step adds a compile-time constant to the tile's base
                    // descriptor (this thread shares its SMSP with ALU-heavy epilogue
                    // warps: few ALU instructions per MMA keep the tensor pipe fed)
                    const uint64_t ad0 = sw128_desc(su32(a16 + ab * C::A16_BYTES));
                    const uint64_t bd0 = sw128_desc(su32(bst + s * C::B_BYTES));
                    const uint32_t dt = tmem + (uint32_t)(buf * BN);
#pragma unroll
                    for (int ks = 0; ks < KA * 4; ++ks) {
                        if (ks < ksteps) {
                            const uint64_t ao = (uint64_t)(((ks >> 2) * (BM * 128) + (ks & 3) * 32) >> 4);
                            const uint64_t bo = (uint64_t)(((ks >> 2) * (BN * 128) + (ks & 3) * 32) >> 4);
                            mma_bf16(dt, ad0 + ao, bd0 + bo, idesc, ks > 0 ? 1u : 0u);
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
        const int quarter = warp & 3;         // TMEM lane quarter this warp may read
        const int grp = e >> 2;               // column group of each center tile
        const int row = quarter * 32 + lane;  // row within the tile
        const float INF = __uint_as_float(0x7F800000u);
        // kValMask as a runtime value: held in a register, the column is then the
        // one immediate of a single logic op per key
        const uint32_t vmask = p.vmask;
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
                // two independent top-2 chains (alternate column pairs), merged per tile
                float k1a = INF, k2a = INF, k1b = INF, k2b = INF;
                const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * BN + grp * C::GW);
                static_assert(C::CHUNKS <= 2, "one load round per tile");
#pragma unroll
                for (int c = 0; c < C::CHUNKS; c += 2) {
                    uint32_t r[2][32];
                    tmem_ld32(tbase + c * 32, r[0]);
                    if (c + 1 < C::CHUNKS) tmem_ld32(tbase + (c + 1) * 32, r[1]);
                    tmem_wait_ld();
                    // the warp's columns are in registers: the accumulator buffer goes
                    // back to the MMA warp now, so the next tile's MMAs overlap this
                    // warp's work on these values
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sm.acc_empty[buf]);
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {
                        if (c + cc >= C::CHUNKS) break;
#pragma unroll
                        for (int q = 0; q < 32; q += 8) {
                            // value-only minimum of each pair of adjacent centers, then a
                            // key: the pair minimum with the pair's number within the
                            // group in the low mantissa bits (a compile-time constant)
                            const uint32_t pc = (uint32_t)(((c + cc) * 32 + q) >> 1);
                            const float m0 = fminf(__uint_as_float(r[cc][q]), __uint_as_float(r[cc][q + 1]));
                            const float m1 = fminf(__uint_as_float(r[cc][q + 2]), __uint_as_float(r[cc][q + 3]));
                            const float m2 = fminf(__uint_as_float(r[cc][q + 4]), __uint_as_float(r[cc][q + 5]));
                            const float m3 = fminf(__uint_as_float(r[cc][q + 6]), __uint_as_float(r[cc][q + 7]));
                            const float a = __uint_as_float((__float_as_uint(m0) & vmask) | pc);
                            const float b = __uint_as_float((__float_as_uint(m1) & vmask) | (pc + 1));
                            const float e = __uint_as_float((__float_as_uint(m2) & vmask) | (pc + 2));
                            const float f = __uint_as_float((__float_as_uint(m3) & vmask) | (pc + 3));
                            const float loa = fminf(a, b), hia = fmaxf(a, b);
                            const float lob = fminf(e, f), hib = fmaxf(e, f);
                            k2a = min3f(fmaxf(k1a, loa), k2a, hia);
                            k1a = fminf(k1a, loa);
                            k2b = min3f(fmaxf(k1b, lob), k2b, hib);
                            k1b = fminf(k1b, lob);
                        }
                    }
                }
                const float k1 = fminf(k1a, k1b);
                const float k2 = min3f(fmaxf(k1a, k1b), k2a, k2b);
                if (k1 < K1) { K2 = fminf(K1, k2); K1 = k1; T1 = t; }
                else K2 = min3f(K2, k1, k2);
            }
            if (!ok) break;
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
                J1 = T1 * BN + 2 * (int)(__float_as_uint(K1) & ~kValMask);
#pragma unroll
                for (int q = 0; q < kGroups - 1; ++q) {
                    const float m1v = __uint_as_float(__float_as_uint(o1[q]) & kValMask);
                    const float k1v = __uint_as_float(__float_as_uint(K1) & kValMask);
                    const int oj = ot[q] * BN + (q + 1) * C::GW + 2 * (int)(__float_as_uint(o1[q]) & ~kValMask);
                    if (m1v < k1v || (m1v == k1v && oj < J1)) { K2 = min3f(K1, o2[q], K2); K1 = o1[q]; J1 = oj; }
                    else K2 = min3f(K2, o1[q], o2[q]);
                }
            }
            // ---- the best pair and the best screened value outside it; the refine
            // computes the pair exactly and decides whether it is certain
            const int64_t R = (int64_t)rt * BM + row;
            if (R < n) {
                p.cand1[R] = J1 < cnt ? begin + J1 : -1;
                p.v2[R] = __uint_as_float(__float_as_uint(K2) & kValMask);
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

size_t tc_anchor_scratch_doubles(int d) { return (size_t)kAnchorBlocks * d; }

cudaError_t launch_anchor(const float *X, int64_t n, int d, double *scratch, float *anchor, cudaStream_t s) {
    anchor_partial_kernel<<<kAnchorBlocks, 256, 0, s>>>(X, n, d, scratch);
    anchor_final_kernel<<<d, 256, 0, s>>>(scratch, n, d, anchor);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_prep_points(const float *X, int64_t n, int d, int split, const float *anchor, uint8_t *img,
                               float *xnorm, cudaStream_t s) {
    const int64_t n_pad = ((n + BM - 1) / BM) * BM;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n_pad / BM, 8192));
    const size_t sm = sizeof(float) * BM * (size_t)d;
    cudaError_t e = cudaFuncSetAttribute(prep_points_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    prep_points_kernel<<<grid, BM, sm, s>>>(X, n, n_pad, d, split, tc_katoms(d, split), anchor, img, xnorm);
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
    // x' = fl(x - a), c' = fl(c - a) move each coordinate by at most 2^-24 of its
    // size, so d(x', c') is within 2^-24 (||x'|| + ||c'||) of d(x, c) and d^2
    // within 2^-22 (||x'||^2 + ||c'||^2)
    const double move = std::ldexp(1.0, -22);
    const double en = 1.25 * (norm + acc + move);
    return Bound{(float)ep, (float)en};
}

cudaError_t launch_prep_centers(const float *C, int d, int split, const DevState *st, int cnt_static, int round_mode,
                                int cap_rows, const float *anchor, uint8_t *img, unsigned int *cmax_bits,
                                cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(cmax_bits, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const int KA = tc_katoms(d, split), BN = tc_block_n(d, split);
    const int rows = ((cap_rows + BN - 1) / BN) * BN;
    if (d > kPrepMaxD) return cudaErrorInvalidValue;
    const int grid = std::max(1, std::min((rows + 7) / 8, 4096));
    prep_centers_kernel<<<grid, 256, 0, s>>>(C, d, split, KA, BN, st, cnt_static, round_mode, anchor, img, cmax_bits);
    count_launches(1);
    return cudaGetLastError();
}

void tc_bound(int d, int split, float *ep, float *en) {
    const Bound b = make_bound(d, split);
    *ep = b.ep;
    *en = b.en;
}

cudaError_t launch_nearest_tc(TcParams p, int mode_round, int num_sms, cudaStream_t s) {
    p.ksteps = tc_ksteps(p.d, p.split);
    p.vmask = kValMask;
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
