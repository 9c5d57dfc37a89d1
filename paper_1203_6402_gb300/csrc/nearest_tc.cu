// nearest_tc.cu -- operand preparation and host side of the tcgen05 screening
// passes (Alg. 2 step 5, Sec. 3.3; Lloyd's assignment, Sec. 3.1).  The pass itself
// is the template of nearest_tc_kernel.cuh, instantiated per operand format in
// nearest_tc_<format>.cu.
//
// The A operand (points) is encoded once per context by prep_points_kernel into a
// swizzled image of X (one contiguous block per 128-row tile) together with
// ||x'||^2 (and, for FP8, the per-row power-of-two scale); the B operand (centers)
// is encoded per pass by prep_centers_kernel (norms in K columns) or
// prep_centers_ne_kernel (one CTA per center tile: ||c'||^2 per center and, for
// FP8, the tile's power-of-two scale).
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <float.h>

#include <algorithm>
#include <cmath>

#include "nearest_tc_kernel.cuh"

namespace kmp {
namespace tc {

// per-format dispatchers (nearest_tc_<format>.cu)
cudaError_t dispatch_bf16(const TcParams &p, int mode_round, int epi, int KA, int grid, cudaStream_t s);
cudaError_t dispatch_bf16x3(const TcParams &p, int mode_round, int epi, int KA, int grid, cudaStream_t s);
cudaError_t dispatch_bf16n(const TcParams &p, int mode_round, int epi, int KA, int grid, cudaStream_t s);
cudaError_t dispatch_fp8(const TcParams &p, int mode_round, int epi, int KA, int grid, cudaStream_t s);

// byte offset of 16-byte chunk c of row r in a K-atom of an SW128 tile
__host__ __device__ __forceinline__ uint32_t sw128_off(int r, int c) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

// ------------------------------------------------------------------ operand encoding
__device__ __forceinline__ __nv_bfloat16 bf(float v) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ uint8_t e4m3(float v) {
    return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

// smallest power of two s with amax / s <= 448 (the largest finite e4m3 value);
// 1 when amax is 0
__device__ __forceinline__ float fp8_scale(float amax) {
    if (!(amax > 0.f)) return 1.f;
    int e;
    const float m = frexpf(amax / 448.f, &e);   // amax / 448 = m 2^e, m in [0.5, 1)
    if (m == 0.5f) e -= 1;
    return ldexpf(1.f, e);
}

struct Enc {
    int d;
    int fmt;
    const float *a;   // anchor: x' = fl(x - a), c' = fl(c - a); nullptr: the row is already moved
};

// x'_q = fl(x_q - a_q)
__device__ __forceinline__ float moved(const Enc &e, const float *x, int q) {
    return e.a ? __fsub_rn(x[q], e.a[q]) : x[q];
}

// element k of a BF16 A (point) row
__device__ __forceinline__ __nv_bfloat16 a_elem(const Enc &e, const float *x, int k) {
    const int d = e.d;
    if (e.fmt == FMT_BF16N) return k < d ? bf(moved(e, x, k)) : bf(0.f);
    if (e.fmt == FMT_BF16) {
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

// element k of a BF16 B (center) row.  Pad rows (no center) get a huge FINITE squared
// norm, so their screened value stays finite: a key built from +inf would become
// a NaN once the column bits are or-ed into its mantissa.
__device__ __forceinline__ __nv_bfloat16 b_elem(const Enc &e, const float *c, float cn_hi, float cn_lo, bool pad, int k) {
    const int d = e.d;
    if (e.fmt == FMT_BF16N) return (!pad && k < d) ? bf(moved(e, c, k)) : bf(0.f);
    const int base = e.fmt == FMT_BF16X3 ? 3 * d : d;
    if (pad) return k == base ? bf(kPadNorm) : bf(0.f);
    if (e.fmt == FMT_BF16) {
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

// 16 e4m3 codes of elements k0 .. k0+15 of a moved row scaled by inv (a power of two)
__device__ __forceinline__ uint4 pack16_e4m3(const float *row, int d, int k0, float inv, bool pad) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint32_t v = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int k = k0 + 4 * i + b;
            const uint8_t code = (!pad && k < d) ? e4m3(row[k] * inv) : (uint8_t)0;
            v |= (uint32_t)code << (8 * b);
        }
        w[i] = v;
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// ------------------------------------------------------------------ center tiles
// Norms in K columns (BF16, BF16X3): one warp per padded center row: the moved row
// c' = fl(c - anchor) is staged in shared memory, lane 0 sums ||c'||^2 (FP32,
// ascending) and records the running max of ||c'||, and lanes 0 .. 8 KA - 1 build
// the row's 16-byte chunks of the B image [tile][katom][BN rows][128 B] in parallel.
constexpr int kPrepMaxD = 384;

__global__ void __launch_bounds__(256) prep_centers_kernel(const float *__restrict__ C, int d, int fmt, int KA, int BN,
                                                           const DevState *st, int cnt_static, int round_mode,
                                                           const float *__restrict__ anchor, uint8_t *__restrict__ img,
                                                           unsigned int *cmax_bits) {
    __shared__ float crow[8][kPrepMaxD];
    const int begin = round_mode ? st->batch_begin : 0;
    const int cnt = round_mode ? st->batch_cnt : cnt_static;
    const int rows = ((cnt + BN - 1) / BN) * BN;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const Enc em{d, fmt, nullptr};   // the staged row is already moved
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

// Norms in the epilogue (BF16N, FP8): one CTA per center tile of BN rows.  FP8
// first finds the tile's largest |c'_q| and its power-of-two scale s_t (tscale[t]);
// then one warp per row stages c', sums ||c'||^2 (FP32: lane-strided partial
// sums, then a fixed shuffle tree) into ncol (pad rows: kPadNorm), records the
// running max of ||c'|| and builds the row's 16-byte chunks: BF16 c', or
// e4m3(c' / s_t).
__global__ void __launch_bounds__(256) prep_centers_ne_kernel(const float *__restrict__ C, int d, int fmt, int KA,
                                                              int BN, const DevState *st, int cnt_static,
                                                              int round_mode, const float *__restrict__ anchor,
                                                              uint8_t *__restrict__ img, float *__restrict__ ncol,
                                                              float *__restrict__ tscale, unsigned int *cmax_bits) {
    __shared__ float crow[8][kPrepMaxD];
    __shared__ float wmax[8];
    const int begin = round_mode ? st->batch_begin : 0;
    const int cnt = round_mode ? st->batch_cnt : cnt_static;
    const int t = blockIdx.x;
    if (t * BN >= cnt) return;   // uniform per block: past the last tile
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j0 = t * BN, j1 = min(cnt, j0 + BN);
    float inv = 1.f;
    if (fmt == FMT_FP8) {
        float am = 0.f;
        for (int j = j0 + w; j < j1; j += 8) {
            const float *c = C + (int64_t)(begin + j) * d;
            for (int q = lane; q < d; q += 32) am = fmaxf(am, fabsf(__fsub_rn(c[q], anchor[q])));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
        if (lane == 0) wmax[w] = am;
        __syncthreads();
        float tm = 0.f;
        for (int i = 0; i < 8; ++i) tm = fmaxf(tm, wmax[i]);
        const float s = fp8_scale(tm);
        inv = 1.f / s;   // exact: s is a power of two
        if (threadIdx.x == 0) tscale[t] = s;
    } else if (threadIdx.x == 0) {
        tscale[t] = 1.f;
    }
    const Enc em{d, fmt, nullptr};
    float *cr = crow[w];
    uint8_t *tile = img + (size_t)t * KA * BN * 128;
    for (int jj = w; jj < BN; jj += 8) {   // uniform per warp
        const int j = j0 + jj;
        const bool pad = j >= cnt;
        if (!pad) {
            const float *c = C + (int64_t)(begin + j) * d;
            for (int q = lane; q < d; q += 32) cr[q] = __fsub_rn(c[q], anchor[q]);
        }
        __syncwarp();
        float part = 0.f;
        if (!pad)
            for (int q = lane; q < d; q += 32) part = __fmaf_rn(cr[q], cr[q], part);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if (lane == 0) {
            ncol[j] = pad ? kPadNorm : part;
            if (!pad) atomicMax(cmax_bits, __float_as_uint(sqrtf(part)));
        }
        if (lane < KA * 8) {
            const int a = lane >> 3, ch = lane & 7;
            uint4 u;
            if (fmt == FMT_FP8) {
                u = pack16_e4m3(cr, d, a * 128 + ch * 16, inv, pad);
            } else {
                __nv_bfloat16 v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = b_elem(em, cr, 0.f, 0.f, pad, a * 64 + ch * 8 + q);
                u = pack8(v);
            }
            *reinterpret_cast<uint4 *>(tile + (size_t)a * BN * 128 + sw128_off(jj, ch)) = u;
        }
        __syncwarp();   // the staged row is read before the next one overwrites it
    }
}

// One CTA per 128-row tile of the A image [row tile][katom][128 rows][128 B]: the
// tile's rows (contiguous in X) come into shared memory with coalesced loads; then
// eight consecutive threads build the eight 16-byte chunks of one row segment of an
// atom (position p of row r holds logical chunk p ^ (r & 7)), so the stores are
// coalesced too; thread r sums ||x'||^2 of row r (FP32, ascending; x' = x - anchor)
// and, for FP8, finds the row's largest |x'_q| and its power-of-two scale s_x.
__global__ void __launch_bounds__(128) prep_points_kernel(const float *__restrict__ X, int64_t n, int64_t n_pad, int d,
                                                          int fmt, int KA, const float *__restrict__ anchor,
                                                          uint8_t *__restrict__ img, float *__restrict__ xnorm,
                                                          float *__restrict__ xscale) {
    extern __shared__ float xsm[];   // BM x d moved rows
    __shared__ float inv_s[BM];
    const int64_t ntile = n_pad / BM;
    for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int64_t r0 = t * BM;
        const int nr = (int)max((int64_t)0, min((int64_t)BM, n - r0));
        __syncthreads();   // the previous tile's readers are done
        for (int f = threadIdx.x; f < nr * d; f += BM) xsm[f] = __fsub_rn(__ldg(X + r0 * d + f), anchor[f % d]);
        __syncthreads();
        {
            const int r = threadIdx.x;
            float xn = 0.f, am = 0.f;
            if (r < nr)
                for (int q = 0; q < d; ++q) {
                    const float v = xsm[r * d + q];
                    xn = __fmaf_rn(v, v, xn);
                    am = fmaxf(am, fabsf(v));
                }
            xnorm[r0 + r] = xn;
            const float s = fmt == FMT_FP8 ? fp8_scale(am) : 1.f;
            if (fmt == FMT_FP8) xscale[r0 + r] = s;
            inv_s[r] = 1.f / s;
        }
        __syncthreads();
        uint8_t *tile = img + (size_t)t * KA * BM * 128;
        const int pos = threadIdx.x & 7;
        const Enc em{d, fmt, nullptr};   // the staged rows are already moved
        for (int a = 0; a < KA; ++a)
            for (int r = threadIdx.x >> 3; r < BM; r += BM / 8) {
                const int ch = pos ^ (r & 7);
                uint4 u;
                if (fmt == FMT_FP8) {
                    u = pack16_e4m3(xsm + r * d, d, a * 128 + ch * 16, inv_s[r], r >= nr);
                } else {
                    __nv_bfloat16 v[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[q] = r < nr ? a_elem(em, xsm + r * d, a * 64 + ch * 8 + q) : bf(0.f);
                    u = pack8(v);
                }
                *reinterpret_cast<uint4 *>(tile + (size_t)a * BM * 128 + r * 128 + pos * 16) = u;
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

// ------------------------------------------------------------------ gather of undecided rows
// Thread per (listed row i, 16-byte chunk): chunk c of image row rows[i] is copied
// to row i of the compact image (both in the SW128 layout).  The first thread of a
// row also copies its scale and sets the list threshold
//     thr = ub - ||x'||^2 + T,   T = 1.02 (Eo + 2 W ub),
// where ub is an exact FP32 upper bound of the distance that decides the row (the
// current center or the pair's best in a round, the pair's best in Lloyd), W the
// FP32 tie window and Eo the screening bound for centers that can matter
// (||c'|| <= ||x'|| + sqrt(ub (1 + 2 W)); farther ones exceed ub (1 + 2 W) by the
// triangle inequality).  Any center left off the list then has an exact distance
// above ub (1 + 2 W) (see the list refine).
// list threshold of a row whose nearest distance is at most u (exact FP32): every
// center whose screened value exceeds it is provably farther than the nearest one
// (twice the screening bound plus the FP32 tie window); +inf without a bound
__device__ __forceinline__ float list_threshold(float u, float xnorm, float cmax, float ep, float en, float ec,
                                                float W) {
    const float xn = fmaxf(xnorm, 0.f);
    const float X = sqrtf(xn);
    float t = __uint_as_float(0x7F800000u);
    if (u < FLT_MAX) {
        const float lim = fmaxf(u, 0.f) * (1.f + 2.f * W);
        const float ceff = fminf(cmax, X + sqrtf(lim));
        const float Eo = ep * X * ceff + en * (xn + ceff * ceff) + ec * X * cmax;
        t = u - xn + 1.02f * (Eo + 2.f * W * fmaxf(u, 0.f)) + 1e-30f;
    }
    return t;
}

__global__ void __launch_bounds__(256) row_thresholds_kernel(const float *__restrict__ ub, int64_t n, int d,
                                                             const float *__restrict__ xnorm,
                                                             const unsigned int *cmax_bits, float ep, float en,
                                                             float ec, float *__restrict__ thr) {
    const float W = fp32_tie_window(d);
    const float cmax = __uint_as_float(*cmax_bits);
    for (int64_t R = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; R < n; R += (int64_t)gridDim.x * blockDim.x)
        thr[R] = list_threshold(ub[R], xnorm[R], cmax, ep, en, ec, W);
}

__global__ void __launch_bounds__(256) gather_rows_kernel(const uint8_t *__restrict__ img,
                                                          const float *__restrict__ xscale, int d, int KA,
                                                          const int32_t *__restrict__ rows, const int *cnt,
                                                          const float *__restrict__ ub, const float *__restrict__ xnorm,
                                                          const unsigned int *cmax_bits, float ep, float en, float ec,
                                                          uint8_t *__restrict__ cimg, float *__restrict__ cscale,
                                                          float *__restrict__ thr) {
    const int64_t nf = *cnt;
    const int per_row = KA * 8;
    const float W = fp32_tie_window(d);
    const float cmax = __uint_as_float(*cmax_bits);
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nf * per_row;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = f / per_row;
        const int a = (int)((f % per_row) >> 3), ch = (int)(f & 7);
        const int64_t R = rows[i];
        const uint8_t *src = img + (size_t)(R / BM) * KA * BM * 128 + (size_t)a * BM * 128 + sw128_off((int)(R % BM), ch);
        uint8_t *dst = cimg + (size_t)(i / BM) * KA * BM * 128 + (size_t)a * BM * 128 + sw128_off((int)(i % BM), ch);
        *reinterpret_cast<uint4 *>(dst) = __ldg(reinterpret_cast<const uint4 *>(src));
        if (a == 0 && ch == 0) {
            cscale[i] = xscale ? xscale[R] : 1.f;
            thr[i] = list_threshold(ub[R], xnorm[R], cmax, ep, en, ec, W);
        }
    }
}

// ------------------------------------------------------------------ host side
int tc_format(int precision, int d) {
    if (precision == KMPAR_BF16X3) return FMT_BF16X3;
    if (precision == KMPAR_FP8E4M3) return FMT_FP8;
    if (precision == KMPAR_BF16)
        // the two norm columns would add a K atom: keep K = d and add the norms in the epilogue
        return ((d + 2 + 63) / 64 > (d + 63) / 64) ? FMT_BF16N : FMT_BF16;
    return -1;
}

static int k_bytes(int d, int fmt) {
    switch (fmt) {
        case FMT_BF16: return 2 * (d + 2);
        case FMT_BF16X3: return 2 * (3 * d + 2);
        case FMT_BF16N: return 2 * d;
        default: return d;   // FMT_FP8
    }
}

int tc_katoms(int d, int fmt) { return (k_bytes(d, fmt) + 127) / 128; }
int tc_ksteps(int d, int fmt) { return (k_bytes(d, fmt) + 31) / 32; }
int tc_block_n(int d, int fmt) { return tc_katoms(d, fmt) <= 2 ? 256 : 128; }
bool tc_norms_in_epilogue(int fmt) { return fmt == FMT_BF16N || fmt == FMT_FP8; }
// the refine and fix-up kernels size their shared-memory rows for d <= 190
bool tc_supported(int d, int fmt) { return fmt >= 0 && d >= 1 && d <= 190 && tc_katoms(d, fmt) <= 3; }

size_t tc_points_image_bytes(int d, int fmt, int64_t n) {
    const int64_t tiles = (n + BM - 1) / BM;
    return (size_t)tiles * tc_katoms(d, fmt) * BM * 128;
}

size_t tc_anchor_scratch_doubles(int d) { return (size_t)kAnchorBlocks * d; }

cudaError_t launch_anchor(const float *X, int64_t n, int d, double *scratch, float *anchor, cudaStream_t s) {
    anchor_partial_kernel<<<kAnchorBlocks, 256, 0, s>>>(X, n, d, scratch);
    anchor_final_kernel<<<d, 256, 0, s>>>(scratch, n, d, anchor);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_prep_points(const float *X, int64_t n, int d, int fmt, const float *anchor, uint8_t *img,
                               float *xnorm, float *xscale, cudaStream_t s) {
    const int64_t n_pad = ((n + BM - 1) / BM) * BM;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n_pad / BM, 8192));
    const size_t sm = sizeof(float) * BM * (size_t)d;
    cudaError_t e = cudaFuncSetAttribute(prep_points_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    prep_points_kernel<<<grid, BM, sm, s>>>(X, n, n_pad, d, fmt, tc_katoms(d, fmt), anchor, img, xnorm, xscale);
    count_launches(1);
    return cudaGetLastError();
}

// Screening error bound E(x, c) >= |s~(x, c) - s(x, c)| (Sec. 3.1 distances,
// s = ||c'||^2 - 2 x'.c'), as E = ep ||x'|| ||c'|| + en (||x'||^2 + ||c'||^2)
// + ec ||x'|| max ||c'||.  Per-element rounding: BF16 u = 2^-8 relative; e4m3
// u = 2^-4 relative plus at most 2^-10 absolute (half its subnormal spacing) in
// scaled units, the scales being at most 2 max|x'_q| / 448 <= 2 ||x'|| / 448
// (rows) and 2 max ||c'|| / 448 (center tiles).  The tensor core's FP32
// accumulation order is not documented, so its error is bounded generously by
// K 2^-23 of the sum of |products|.  en collects the FP32 norm sums, the split of
// ||c'||^2 into two BF16 columns (BF16, BF16X3) or the epilogue FMA (BF16N, FP8),
// and the anchor move (fl(x - a) moves d^2 by at most 2^-22 (||x'||^2 + ||c'||^2)).
struct Bound {
    float ep, en, ec;
};

Bound make_bound(int d, int fmt) {
    const int K = tc_ksteps(d, fmt) * 32 / (fmt == FMT_FP8 ? 1 : 2);   // K elements executed
    const double acc = K * std::ldexp(1.0, -23);
    const double move = std::ldexp(1.0, -22);
    const double nsum = (d + 2) * std::ldexp(1.0, -24);
    double ep, en, ec = 0.0;
    if (fmt == FMT_FP8) {
        const double u = 1.0 / 16.0, eta = std::ldexp(1.0, -10);
        const double sc = 2.0 / 448.0;                          // scale / norm bound
        const double sub = eta * std::sqrt((double)d) * sc * (1.0 + u);
        // the sum of |products| is at most (1 + u)^2 ||x'|| ||c'|| (plus the scaled
        // subnormal terms), so the accumulation adds acc (1 + u)^2 < 1.2 acc of it
        ep = 2.0 * ((2.0 * u + u * u) + sub + 1.2 * acc);
        ec = 2.0 * (sub + d * eta * eta * sc * sc) * (1.0 + 1.2 * acc);
        en = nsum + 2.0 * std::ldexp(1.0, -24) + move;
    } else {
        const double u = 1.0 / 256.0;
        ep = fmt == FMT_BF16X3 ? 2.0 * (3.0 * u * u + 3.0 * u * u * u) : 2.0 * (2.0 * u + u * u);
        ep += 2.0 * acc * 1.1;
        const double norm = (fmt == FMT_BF16N) ? 2.0 * std::ldexp(1.0, -24) : u * u;
        en = norm + nsum + acc + move;
    }
    return Bound{(float)(1.25 * ep), (float)(1.25 * en), (float)(1.25 * ec)};
}

int tc_center_tiles(int d, int fmt, int cap_rows) {
    const int BN = tc_block_n(d, fmt);
    return (cap_rows + BN - 1) / BN;
}

cudaError_t launch_prep_centers(const float *C, int d, int fmt, const DevState *st, int cnt_static, int round_mode,
                                int cap_rows, const float *anchor, uint8_t *img, float *ncol, float *tscale,
                                unsigned int *cmax_bits, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(cmax_bits, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const int KA = tc_katoms(d, fmt), BN = tc_block_n(d, fmt);
    if (d > kPrepMaxD) return cudaErrorInvalidValue;
    const int tiles = tc_center_tiles(d, fmt, cap_rows);
    if (tc_norms_in_epilogue(fmt)) {
        prep_centers_ne_kernel<<<std::max(1, tiles), 256, 0, s>>>(C, d, fmt, KA, BN, st, cnt_static, round_mode,
                                                                   anchor, img, ncol, tscale, cmax_bits);
    } else {
        const int grid = std::max(1, std::min((tiles * BN + 7) / 8, 4096));
        prep_centers_kernel<<<grid, 256, 0, s>>>(C, d, fmt, KA, BN, st, cnt_static, round_mode, anchor, img,
                                                 cmax_bits);
    }
    count_launches(1);
    return cudaGetLastError();
}

void tc_bound(int d, int fmt, float *ep, float *en, float *ec) {
    const Bound b = make_bound(d, fmt);
    *ep = b.ep;
    *en = b.en;
    *ec = b.ec;
}

cudaError_t launch_gather_rows(const uint8_t *img, const float *xscale, int d, int fmt, const int32_t *rows,
                               const int *cnt, const float *ub, const float *xnorm, const unsigned int *cmax_bits,
                               float ep, float en, float ec, uint8_t *cimg, float *cscale, float *thr, int grid,
                               cudaStream_t s) {
    gather_rows_kernel<<<grid, 256, 0, s>>>(img, fmt == FMT_FP8 ? xscale : nullptr, d, tc_katoms(d, fmt), rows, cnt,
                                            ub, xnorm, cmax_bits, ep, en, ec, cimg, cscale, thr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_row_thresholds(const float *ub, int64_t n, int d, const float *xnorm,
                                  const unsigned int *cmax_bits, float ep, float en, float ec, float *thr,
                                  cudaStream_t s) {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(4096, (n + 255) / 256));
    row_thresholds_kernel<<<grid, 256, 0, s>>>(ub, n, d, xnorm, cmax_bits, ep, en, ec, thr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_nearest_tc(TcParams p, int mode_round, int epi, int num_sms, cudaStream_t s) {
    p.ksteps = tc_ksteps(p.d, p.fmt);
    p.vmask = kValMask;
    const int KA = tc_katoms(p.d, p.fmt);
    // EPI_LIST: the row count is on the device; every SM takes part
    const int rows = epi == EPI_LIST ? num_sms : (int)((p.n + BM - 1) / BM);
    const int grid = std::max(1, std::min(rows, num_sms));
    switch (p.fmt) {
        case FMT_BF16: return dispatch_bf16(p, mode_round, epi, KA, grid, s);
        case FMT_BF16X3: return dispatch_bf16x3(p, mode_round, epi, KA, grid, s);
        case FMT_BF16N: return dispatch_bf16n(p, mode_round, epi, KA, grid, s);
        case FMT_FP8: return dispatch_fp8(p, mode_round, epi, KA, grid, s);
    }
    return cudaErrorInvalidValue;
}

size_t tc_image_bytes(int d, int fmt, int cap_rows) {
    const int KA = tc_katoms(d, fmt), BN = tc_block_n(d, fmt);
    return (size_t)tc_center_tiles(d, fmt, cap_rows) * KA * BN * 128;
}

}  // namespace tc
}  // namespace kmp
