// round_simt.cu -- the per-round data-parallel pass of k-means|| (Alg. 2 steps
// 1-2, 4-5 of Bahmani et al., Sec. 3.3) and the nearest-center scan that Lloyd's
// iteration and phi_X(C) (Sec. 3.1) reuse, on CUDA cores in exact FP32.
//
// Kernels:
//   pick_first_kernel   Alg. 2 step 1: i0 = floor(u n), row gathered as candidate 0
//   nearest_kernel      d^2(x, C') for the batch C' (or all k centers), top-2 per
//                       row, FP64 re-decision of near ties, D^2/idx/labels update,
//                       per-block FP64 partial of phi
//   sample_kernel       Alg. 2 step 4: p = min(1, l D^2/phi), Philox draw,
//                       warp-aggregated atomic append
//   sort_batch_kernel   ascending order of the round's draws (one CTA, bitonic)
//   gather_kernel       candidate rows copied out of X
//   sum_f64_kernel      fixed-order FP64 sum of per-block partials
#include <float.h>

#include <algorithm>

#include "kmpar_internal.cuh"

namespace kmp {

constexpr int kNearThreads = 128;

enum { MODE_FIRST = 0, MODE_ROUND = 1, MODE_ASSIGN = 2 };

struct NearestParams {
    const float *X;
    int64_t n;
    int d;
    const float *C;        // center rows, stride d
    int c_begin, c_cnt;    // ASSIGN: static range; FIRST/ROUND: taken from st
    const DevState *st;
    float *D2;             // FIRST: out; ROUND: in/out
    int32_t *idx;          // FIRST: out; ROUND: in/out
    int32_t *labels;       // ASSIGN: out (nullable)
    const int32_t *prev;   // ASSIGN: previous labels (nullable)
    int *changed;          // ASSIGN: +number of labels != prev (nullable)
    double *partials;      // per-block FP64 sum of the stored distances (nullable)
    unsigned long long *fp64_cnt, *wide_cnt;
    const int32_t *rows;   // nullable: process only these rows (the tensor pass's fix-up list)
    const int *rows_cnt;   // number of entries in rows
    float *dmin;           // ASSIGN: per-row exact d^2 of the chosen center (nullable)
};

// lexicographic (value, index) improvement
__device__ __forceinline__ void take_if_better(double v, int j, double &best, int &bj) {
    if (v < best || (v == best && j < bj)) { best = v; bj = j; }
}

template <int DP, int MODE>
__global__ void __launch_bounds__(kNearThreads) nearest_kernel(NearestParams p) {
    constexpr int TC = DP == 0 ? 1 : (DP <= 64 ? 64 : 32);
    constexpr int TILE = DP == 0 ? 4 : TC * DP;
    __shared__ __align__(16) float tile[TILE];
    __shared__ double red[32];
    __shared__ int redi[32];

    const int tid = threadIdx.x;
    int64_t pt = (int64_t)blockIdx.x * kNearThreads + tid;
    bool valid = pt < p.n;
    if (p.rows) {
        const int nrows = *p.rows_cnt;
        if ((int64_t)blockIdx.x * kNearThreads >= nrows) return;   // uniform per block
        valid = pt < nrows;
        pt = valid ? p.rows[pt] : 0;
    }
    const int d = p.d;
    const float *xrow = p.X + (valid ? pt : 0) * (int64_t)d;

    float xr[DP == 0 ? 1 : DP];
    if constexpr (DP > 0) {
#pragma unroll
        for (int q = 0; q < DP; ++q) xr[q] = (valid && q < d) ? __ldg(xrow + q) : 0.f;
    }

    int begin, cnt;
    if constexpr (MODE == MODE_ASSIGN) {
        begin = p.c_begin; cnt = p.c_cnt;
    } else {
        begin = p.st->batch_begin; cnt = p.st->batch_cnt;
    }

    float b1 = FLT_MAX, b2 = FLT_MAX;
    int i1 = -1, i2 = -1;
    for (int t0 = 0; t0 < cnt; t0 += TC) {
        const int nt = min(TC, cnt - t0);
        if constexpr (DP > 0) {
            __syncthreads();
            for (int e = tid; e < TC * DP; e += kNearThreads) {
                const int r = e / DP, q = e - r * DP;
                tile[e] = (r < nt && q < d) ? __ldg(p.C + (int64_t)(begin + t0 + r) * d + q) : 0.f;
            }
            __syncthreads();
        }
        if (valid) {
            for (int r = 0; r < nt; ++r) {
                float acc = 0.f;
                if constexpr (DP > 0) {
                    const float4 *c4 = reinterpret_cast<const float4 *>(tile + r * DP);
#pragma unroll
                    for (int q4 = 0; q4 < DP / 4; ++q4) {
                        const float4 c = c4[q4];
                        float t;
                        t = __fsub_rn(xr[4 * q4 + 0], c.x); acc = __fmaf_rn(t, t, acc);
                        t = __fsub_rn(xr[4 * q4 + 1], c.y); acc = __fmaf_rn(t, t, acc);
                        t = __fsub_rn(xr[4 * q4 + 2], c.z); acc = __fmaf_rn(t, t, acc);
                        t = __fsub_rn(xr[4 * q4 + 3], c.w); acc = __fmaf_rn(t, t, acc);
                    }
                } else {
                    acc = dist2_fp32(xrow, p.C + (int64_t)(begin + t0 + r) * d, d);
                }
                const int j = begin + t0 + r;
                if (acc < b2) {
                    if (acc < b1) { b2 = b1; i2 = i1; b1 = acc; i1 = j; }
                    else { b2 = acc; i2 = j; }
                }
            }
        }
    }

    float stored = 0.f;
    int chg = 0;
    if (valid) {
        const float W = fp32_tie_window(d);
        if constexpr (MODE == MODE_ASSIGN) {
            // a row whose distances are all NaN/inf keeps label 0 (labels stay in range)
            int lab = i1 >= 0 ? i1 : 0;
            stored = b1;
            if (i2 >= 0 && b2 <= b1 + W * b1) {
                // the FP32 order of the two best may differ from the FP64 order
                double best = dist2_fp64(xrow, p.C + (int64_t)i1 * d, d);
                int bj = i1;
                take_if_better(dist2_fp64(xrow, p.C + (int64_t)i2 * d, d), i2, best, bj);
                if (bj == i2) { lab = i2; stored = b2; }
                atomicAdd(p.fp64_cnt, 1ull);
            }
            if (p.labels) p.labels[pt] = lab;
            if (p.dmin) p.dmin[pt] = stored;
            if (p.prev) chg = (p.prev[pt] != lab);
        } else if constexpr (MODE == MODE_FIRST) {
            stored = (i1 >= 0) ? b1 : __int_as_float(0x7f800000);
            p.D2[pt] = stored;
            p.idx[pt] = 0;
        } else {
            const float old = p.D2[pt];
            const int oi = p.idx[pt];
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
                if (in_old) take_if_better(dist2_fp64(xrow, p.C + (int64_t)oi * d, d), oi, best, bj);
                if (in1) take_if_better(dist2_fp64(xrow, p.C + (int64_t)i1 * d, d), i1, best, bj);
                if (in2) take_if_better(dist2_fp64(xrow, p.C + (int64_t)i2 * d, d), i2, best, bj);
                atomicAdd(p.fp64_cnt, 1ull);
                if (in1 && in2) atomicAdd(p.wide_cnt, 1ull);
                if (bj == i1) { win = i1; wv = b1; }
                else if (bj == i2) { win = i2; wv = b2; }
            } else if (i1 >= 0 && b1 < old) {
                win = i1; wv = b1;
            }
            if (win >= 0) {
                p.D2[pt] = wv;
                p.idx[pt] = win;
                stored = wv;
            } else {
                stored = old;
            }
        }
    }

    const double s = block_sum_f64(valid ? (double)stored : 0.0, red);
    if (tid == 0 && p.partials) p.partials[blockIdx.x] = s;
    if constexpr (MODE == MODE_ASSIGN) {
        if (p.changed) {
            int c = warp_sum_i32(chg);
            __syncthreads();
            if ((tid & 31) == 0) redi[tid >> 5] = c;
            __syncthreads();
            if (tid == 0) {
                int tot = 0;
                for (int i = 0; i < kNearThreads / 32; ++i) tot += redi[i];
                if (tot) atomicAdd(p.changed, tot);
            }
        }
    }
}

template <int MODE>
static cudaError_t launch_nearest_mode(const NearestParams &p, cudaStream_t s) {
    const int grid = (int)((p.n + kNearThreads - 1) / kNearThreads);   // p.n = rows capacity for row lists
    const int d = p.d;
#define KMP_NEAREST_CASE(DPV)                                              \
    if (d <= DPV) {                                                         \
        nearest_kernel<DPV, MODE><<<grid, kNearThreads, 0, s>>>(p);          \
        count_launches(1);                                                   \
        return cudaGetLastError();                                           \
    }
    KMP_NEAREST_CASE(4)
    KMP_NEAREST_CASE(8)
    KMP_NEAREST_CASE(16)
    KMP_NEAREST_CASE(32)
    KMP_NEAREST_CASE(48)
    KMP_NEAREST_CASE(64)
    KMP_NEAREST_CASE(96)
    KMP_NEAREST_CASE(128)
#undef KMP_NEAREST_CASE
    nearest_kernel<0, MODE><<<grid, kNearThreads, 0, s>>>(p);
    count_launches(1);
    return cudaGetLastError();
}

int assign_num_partials(int64_t n, int) { return (int)((n + kNearThreads - 1) / kNearThreads); }

// ------------------------------------------------------------------ init
__global__ void pick_first_kernel(const float *X, int64_t n, int d, uint64_t seed, DevState *st,
                                  int32_t *cand, float *C) {
    __shared__ int64_t s_i0;
    if (threadIdx.x == 0) {
        const double u = uniform53(0, 0, TAG_INIT, seed);
        int64_t i0 = (int64_t)floor(__dmul_rn(u, (double)n));
        if (i0 >= n) i0 = n - 1;
        s_i0 = i0;
        st->i0 = (int32_t)i0;
        cand[0] = (int32_t)i0;
        st->m = 1;
        st->batch_begin = 0;
        st->batch_cnt = 1;
        st->drawn = 0;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < d; q += blockDim.x) C[q] = X[s_i0 * (int64_t)d + q];
}

cudaError_t launch_init_first(Ctx &c) {
    pick_first_kernel<<<1, 128, 0, c.stream>>>(c.X, c.n, c.d, c.seed, c.st, c.cand, c.C);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    NearestParams p{};
    p.X = c.X; p.n = c.n; p.d = c.d; p.C = c.C; p.st = c.st; p.D2 = c.D2; p.idx = c.idx;
    p.partials = c.partials; p.fp64_cnt = &c.st->argmin_fp64; p.wide_cnt = &c.st->argmin_wide;
    e = launch_nearest_mode<MODE_FIRST>(p, c.stream);
    if (e != cudaSuccess) return e;
    return launch_phi_finalize(c, assign_num_partials(c.n, c.d), &c.st->phi, &c.st->phi_hist[0]);
}

// ------------------------------------------------------------------ sampling
__global__ void sample_kernel(const float *__restrict__ D2, const int32_t *__restrict__ idx,
                              const float *__restrict__ X, const float *__restrict__ C, int64_t n, int d,
                              double ell, uint32_t round, uint64_t seed, DevState *st, int32_t *drawn,
                              int cap) {
    const double phi = st->phi;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        bool take = false;
        if (i < n) {
            const float dd = D2[i];
            double pr = 0.0;
            if (phi > 0.0) pr = fmin(1.0, __ddiv_rn(__dmul_rn(ell, (double)dd), phi));
            const double u = uniform53((uint64_t)i, round, TAG_SAMPLE, seed);
            if (dd > 0.f && fabs(u - pr) <= 1e-5) {
                // the FP32 D^2 could decide this draw: use the FP64 distance of the definition
                const double d64 = dist2_fp64(X + i * (int64_t)d, C + (int64_t)idx[i] * d, d);
                pr = fmin(1.0, __ddiv_rn(__dmul_rn(ell, d64), phi));
                atomicAdd(&st->sample_refined, 1ull);
            }
            if (fabs(u - pr) <= 1e-6) atomicAdd(&st->sample_near, 1ull);
            take = u < pr;
        }
        const unsigned mask = __ballot_sync(0xffffffffu, take);
        if (mask) {
            const int leader = __ffs(mask) - 1;
            int b = 0;
            if (lane == leader) b = atomicAdd(&st->drawn, __popc(mask));
            b = __shfl_sync(0xffffffffu, b, leader);
            if (take) {
                const int pos = b + __popc(mask & ((1u << lane) - 1u));
                if (pos < cap) drawn[pos] = (int32_t)i;
                else st->overflow = 1;
            }
        }
    }
}

// one CTA: bitonic sort of this round's draws (ascending point order), appended to
// the candidate list; the batch range is published in st for the next kernels.
__global__ void __launch_bounds__(1024) sort_batch_kernel(const int32_t *drawn, int cap, int round,
                                                          DevState *st, int32_t *cand) {
    extern __shared__ int32_t keys[];
    const int total = st->drawn;
    const int cnt = min(total, cap);
    int P = 1;
    while (P < cnt) P <<= 1;
    for (int e = threadIdx.x; e < P; e += blockDim.x) keys[e] = e < cnt ? drawn[e] : INT_MAX;
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int e = threadIdx.x; e < P; e += blockDim.x) {
                const int o = e ^ stride;
                if (o > e) {
                    const bool asc = (e & size) == 0;
                    const int a = keys[e], b = keys[o];
                    if ((a > b) == asc) { keys[e] = b; keys[o] = a; }
                }
            }
        }
    }
    __syncthreads();
    const int m0 = st->m;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) cand[m0 + e] = keys[e];
    __syncthreads();
    if (threadIdx.x == 0) {
        st->batch_begin = m0;
        st->batch_cnt = cnt;
        st->m = m0 + cnt;
        st->round_added[round - 1] = total;
        st->drawn = 0;
    }
}

__global__ void gather_kernel(const float *__restrict__ X, int d, const DevState *st, const int32_t *cand,
                              float *C) {
    const int begin = st->batch_begin, cnt = st->batch_cnt;
    const int64_t total = (int64_t)cnt * d;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / d;
        const int q = (int)(e - r * d);
        C[(begin + r) * d + q] = X[(int64_t)cand[begin + r] * d + q];
    }
}

__global__ void __launch_bounds__(1024) sum_f64_kernel(const double *parts, int nparts, double *out,
                                                      double *copy) {
    __shared__ double sh[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += parts[i];
    const double s = block_sum_f64(v, sh);
    if (threadIdx.x == 0) {
        *out = s;
        if (copy) *copy = s;
    }
}

cudaError_t launch_sum_f64(const double *parts, int nparts, double *out, double *copy, cudaStream_t s) {
    sum_f64_kernel<<<1, 1024, 0, s>>>(parts, nparts, out, copy);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_phi_finalize(Ctx &c, int nparts, double *out, double *hist_slot) {
    return launch_sum_f64(c.partials, nparts, out, hist_slot, c.stream);
}

cudaError_t launch_round(Ctx &c, int round) {
    cudaError_t e;
    if (c.sampling == 1) {
        if ((e = launch_sample_exact(c, round)) != cudaSuccess) return e;
    } else {
        const int sgrid = c.num_sms * 8;
        sample_kernel<<<sgrid, 256, 0, c.stream>>>(c.D2, c.idx, c.X, c.C, c.n, c.d, c.ell, (uint32_t)round,
                                                   c.seed, c.st, c.drawn, c.cap_round);
        count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    int P = 1;
    while (P < c.cap_round) P <<= 1;
    sort_batch_kernel<<<1, 1024, P * sizeof(int32_t), c.stream>>>(c.drawn, c.cap_round, round, c.st, c.cand);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t gtot = (int64_t)c.cap_round * c.d;
    const int ggrid = (int)std::min<int64_t>((gtot + 255) / 256, (int64_t)c.num_sms * 16);
    gather_kernel<<<ggrid, 256, 0, c.stream>>>(c.X, c.d, c.st, c.cand, c.C);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    count_launches(2);
    return launch_round_distance(c, round);
}

cudaError_t launch_sum_rows(const float *v, int64_t n, double *partials, int max_parts, double *out, double *copy,
                            cudaStream_t s);

// Alg. 2 step 5: D^2/idx against the batch just appended, then phi
cudaError_t launch_round_distance(Ctx &c, int round) {
    cudaError_t e;
    if (c.precision != KMPAR_FP32) {
        if ((e = launch_tc_pass(c, 1, c.C, 0, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr)) != cudaSuccess)
            return e;
        return launch_sum_rows(c.D2, c.n, c.partials, c.num_partials, &c.st->phi, &c.st->phi_hist[round], c.stream);
    }
    cudaEvent_t ev = nullptr;
    if ((e = timing_begin(c, &ev)) != cudaSuccess) return e;
    NearestParams p{};
    p.X = c.X; p.n = c.n; p.d = c.d; p.C = c.C; p.st = c.st; p.D2 = c.D2; p.idx = c.idx;
    p.partials = c.partials; p.fp64_cnt = &c.st->argmin_fp64; p.wide_cnt = &c.st->argmin_wide;
    if ((e = launch_nearest_mode<MODE_ROUND>(p, c.stream)) != cudaSuccess) return e;
    if ((e = timing_end(c, ev, 0)) != cudaSuccess) return e;
    return launch_phi_finalize(c, assign_num_partials(c.n, c.d), &c.st->phi, &c.st->phi_hist[round]);
}

cudaError_t launch_assign(const float *X, int64_t n, int d, const float *C, int k, int32_t *labels,
                          const int32_t *prev, int *changed, double *partials, int,
                          unsigned long long *fp64_cnt, cudaStream_t s) {
    NearestParams p{};
    p.X = X; p.n = n; p.d = d; p.C = C; p.c_begin = 0; p.c_cnt = k;
    p.labels = labels; p.prev = prev; p.changed = changed; p.partials = partials;
    p.fp64_cnt = fp64_cnt; p.wide_cnt = fp64_cnt;
    return launch_nearest_mode<MODE_ASSIGN>(p, s);
}

// ------------------------------------------------------------------ generator export
__global__ void uniforms_kernel(int64_t count, uint32_t round, uint32_t tag, uint64_t seed, double *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = uniform53((uint64_t)i, round, tag, seed);
}

cudaError_t launch_uniforms(int64_t count, uint32_t round, uint32_t tag, uint64_t seed, double *out,
                            cudaStream_t s) {
    const int grid = (int)std::min<int64_t>((count + 255) / 256, 4096);
    uniforms_kernel<<<grid > 0 ? grid : 1, 256, 0, s>>>(count, round, tag, seed, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace kmp

namespace kmp {
cudaError_t configure_refine_kernels();

cudaError_t configure_round_kernels(int max_sort_pow2) {
    cudaError_t e = cudaFuncSetAttribute(sort_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         max_sort_pow2 * (int)sizeof(int32_t));
    if (e != cudaSuccess) return e;
    return configure_refine_kernels();
}
}  // namespace kmp

// ------------------------------------------------------------------ tensor-core passes
namespace kmp {

// deterministic FP64 sum of a float array: fixed per-block ranges, fixed trees
__global__ void __launch_bounds__(256) sum_rows_kernel(const float *__restrict__ v, int64_t n, int64_t per_block,
                                                      double *partials) {
    __shared__ double sh[32];
    const int64_t b0 = (int64_t)blockIdx.x * per_block;
    const int64_t b1 = min(n, b0 + per_block);
    double acc = 0.0;
    if ((per_block & 3) == 0 && (reinterpret_cast<uintptr_t>(v) & 15u) == 0) {
        // four consecutive values per thread and step, added in index order
        for (int64_t i = b0 + 4 * threadIdx.x; i < b1; i += 4 * blockDim.x) {
            if (i + 4 <= b1) {
                const float4 q = __ldg(reinterpret_cast<const float4 *>(v + i));
                acc += (double)q.x;
                acc += (double)q.y;
                acc += (double)q.z;
                acc += (double)q.w;
            } else {
                for (int64_t j = i; j < b1; ++j) acc += (double)v[j];
            }
        }
    } else {
        for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) acc += (double)v[i];
    }
    const double s = block_sum_f64(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

cudaError_t launch_sum_rows(const float *v, int64_t n, double *partials, int max_parts, double *out, double *copy,
                            cudaStream_t s) {
    int64_t per = 1024;
    int64_t nb = (n + per - 1) / per;
    if (nb > max_parts) {
        per = (n + max_parts - 1) / max_parts;
        nb = (n + per - 1) / per;
    }
    if (nb < 1) nb = 1;
    sum_rows_kernel<<<(int)nb, 256, 0, s>>>(v, n, per, partials);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_sum_f64(partials, (int)nb, out, copy, s);
}

// (value, index) top-2 of the union of two top-2 lists (lowest index on equal values)
__device__ __forceinline__ bool lex_lt(float v, int i, float w, int j) { return v < w || (v == w && i < j); }

__device__ __forceinline__ void top2_merge(float &b1, int &i1, float &b2, int &i2, float c1, int j1, float c2, int j2) {
    if (lex_lt(c1, j1, b1, i1)) {
        // c1 is the new best; second = best of (b1, c2)
        if (lex_lt(b1, i1, c2, j2)) { b2 = b1; i2 = i1; } else { b2 = c2; i2 = j2; }
        b1 = c1; i1 = j1;
    } else if (lex_lt(c1, j1, b2, i2)) {
        b2 = c1; i2 = j1;
    }
}

// The decision for row R once its best and runner-up candidates (b1, i1), (b2, i2)
// have exact FP32 values (i2 = -1: none), taken exactly as nearest_kernel takes
// it.  Lloyd: the label is the best, re-decided in FP64 against the runner-up
// when their FP32 values lie within the tie window.  Round: the current center
// is replaced by the best new candidate when nearer; when two or more of (current,
// best, runner-up) lie within the tie window they are re-decided in FP64, equal
// FP64 values keeping the lower center number.  Returns 1 when a Lloyd label
// changed.
template <int MODE>
__device__ __forceinline__ int decide_top2(const float *__restrict__ X, int d, const float *__restrict__ C, int64_t R,
                                           float b1, int i1, float b2, int i2, float *D2, int32_t *idx,
                                           int32_t *labels, const int32_t *prev, float *dmin,
                                           unsigned long long *fp64_cnt, unsigned long long *wide_cnt) {
    const float W = fp32_tie_window(d);
    const float *xrow = X + R * d;
    if (MODE == MODE_ASSIGN) {
        int lab = i1 != INT_MAX ? i1 : 0;
        float stored = b1;
        if (i2 >= 0 && b2 <= b1 + W * b1) {
            double best = dist2_fp64(xrow, C + (int64_t)i1 * d, d);
            int bj = i1;
            take_if_better(dist2_fp64(xrow, C + (int64_t)i2 * d, d), i2, best, bj);
            if (bj == i2) { lab = i2; stored = b2; }
            atomicAdd(fp64_cnt, 1ull);
        }
        if (labels) labels[R] = lab;
        if (dmin) dmin[R] = stored;
        return (prev && prev[R] != lab) ? 1 : 0;
    } else {
        const float old = D2[R];
        const int oi = idx[R];
        const float m32 = fminf(old, b1);
        const float lim = m32 + W * m32;
        const bool in_old = (oi >= 0) && old <= lim;
        const bool in1 = i1 != INT_MAX && b1 <= lim;
        const bool in2 = i2 >= 0 && b2 <= lim;
        int win = -1;
        float wv = old;
        if ((int)in_old + (int)in1 + (int)in2 >= 2) {
            double best = DBL_MAX;
            int bj = INT_MAX;
            if (in_old) take_if_better(dist2_fp64(xrow, C + (int64_t)oi * d, d), oi, best, bj);
            if (in1) take_if_better(dist2_fp64(xrow, C + (int64_t)i1 * d, d), i1, best, bj);
            if (in2) take_if_better(dist2_fp64(xrow, C + (int64_t)i2 * d, d), i2, best, bj);
            atomicAdd(fp64_cnt, 1ull);
            if (in1 && in2) atomicAdd(wide_cnt, 1ull);
            if (bj == i1) { win = i1; wv = b1; }
            else if (bj == i2) { win = i2; wv = b2; }
        } else if (i1 != INT_MAX && b1 < old) {
            win = i1; wv = b1;
        }
        if (win >= 0) { D2[R] = wv; idx[R] = win; }
        return 0;
    }
}

// screening statistics of a pass: rows screened, rows the pair screening left
// undecided, and (after the list pass) rows that needed the exact scan
__global__ void count_fixups_kernel(const int *fix_cnt, const int *exact_cnt, int64_t n, const int *rows_cnt,
                                    DevState *st) {
    st->screen_fallback += (unsigned long long)*fix_cnt;
    st->screen_rows += (unsigned long long)(rows_cnt ? (int64_t)*rows_cnt : n);
    st->screen_exact += (unsigned long long)(exact_cnt ? *exact_cnt : *fix_cnt);
}

cudaError_t count_fixups(Ctx &c, const int *exact_cnt, const int *rows_cnt = nullptr) {
    count_fixups_kernel<<<1, 1, 0, c.stream>>>(c.fix_cnt, exact_cnt, c.n, rows_cnt, c.st);
    count_launches(1);
    return cudaGetLastError();
}

// the two halves of count_fixups when the undecided rows pass through several stages
__global__ void count_stage_kernel(const int *fallback_cnt, const int *exact_cnt, int64_t n, DevState *st) {
    if (fallback_cnt) {   // the rows the pair screening left, all refined from their own lists
        st->screen_fallback += (unsigned long long)*fallback_cnt;
        st->screen_listed += (unsigned long long)*fallback_cnt;
        st->screen_rows += (unsigned long long)n;
    }
    if (exact_cnt) st->screen_exact += (unsigned long long)*exact_cnt;
}

// Exact FP32 distances and the decision for the rows the tensor screening has
// brought down to one pair of adjacent centers (cand1 = the pair's first center,
// -1: none).  Both centers of the pair get the exact FP32 difference form
// (ascending coordinates, bit-identical to dist2_fp32); the row is certain when
// every center outside the pair is, by the screening bound, beyond the tie window
// of the pair's best exact value.  Certain rows take the CUDA-core decision
// (decide_top2) on the pair; the others go to the fix-up list.
__host__ __device__ __forceinline__ int refine_stride(int d) { return d + ((6 - (d & 3)) & 3); }   // = 2 mod 4

__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

struct ScreenBound {
    const float *xnorm;            // ||x'||^2 per point (x' = x - anchor)
    const unsigned int *cmax_bits; // max ||c'|| of the batch
    const DevState *st;            // ROUND: batch range
    float ep, en, ec;              // E(x, c) = ep ||x'|| ||c'|| + en (||x'||^2 + ||c'||^2) + ec ||x'|| max ||c'||
    int32_t *fix_rows;
    int *fix_cnt;
    float *ub;                     // per listed row: exact FP32 upper bound of its deciding distance
};

// rows whose screening is not certain go to the fix-up list: one atomic per warp
__device__ __forceinline__ void append_fixups(const ScreenBound &sb, bool fix, int64_t R) {
    const unsigned m = __ballot_sync(0xffffffffu, fix);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0) base = atomicAdd(sb.fix_cnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (fix) sb.fix_rows[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)R;
}

// screened values arrive with their low 6 mantissa bits cleared (relative change
// below 2^-17); twice that is allowed for
constexpr float kKeyTrunc = 1.6e-5f;

// The certainty test.  m = the exact FP32 d^2 that decides the row: the pair's
// best in Lloyd, the nearer of the current center and the pair's best in a round
// (a center farther than the current one changes nothing unless it falls in the
// tie window).  v2 = a lower bound of the screened value (s = ||c'||^2 - 2 x'.c')
// of every center not examined exactly.  Such a center c has d^2 = s + ||x'||^2
// >= v2 - E(x, c) + ||x'||^2.  A center with ||c'|| > ||x'|| + sqrt(m (1 + 2W)) is
// farther than m (1 + 2W) by the triangle inequality; every nearer one has
// ||c'|| <= ceff, so E(x, c) <= Eo.  If the bound exceeds m (1 + 2W), no FP32 value
// outside the examined centers can win or fall in the tie window of the best
// (W = fp32_tie_window covers both FP32 errors).
__device__ __forceinline__ bool bound_certain(const ScreenBound &sb, float xnorm, float m, float v2lo, int d) {
    const float xn = fmaxf(xnorm, 0.f);
    const float X = sqrtf(xn);
    const float cmax = __uint_as_float(*sb.cmax_bits);
    const float W = fp32_tie_window(d);
    const float lim = fmaxf(m, 0.f) * (1.f + 2.f * W);
    const float ceff = fminf(cmax, X + sqrtf(lim));
    const float Eo = sb.ep * X * ceff + sb.en * (xn + ceff * ceff) + sb.ec * X * cmax;
    return (v2lo - Eo + xn) > lim + 1e-30f;
}

// the pair screening's v2 arrives key-truncated: lowered by that truncation (stays
// +inf when there is no other center)
__device__ __forceinline__ bool pair_certain(const ScreenBound &sb, float xnorm, float m, float v2, int d) {
    const float v2lo = v2 >= 0.f ? v2 * (1.f - kKeyTrunc) : v2 * (1.f + kKeyTrunc);
    return bound_certain(sb, xnorm, m, v2lo, d);
}

// a lower bound of the real d^2 of every center outside the examined ones, from
// their smallest screened value (key-truncated v2, lowered): v2lo - E + ||x'||^2
// with E at the largest center norm (no triangle-inequality cut: this bound is
// kept for Lloyd's next iteration, where it has to hold for every center)
__device__ __forceinline__ float outside_lb(const ScreenBound &sb, float xnorm, float v2) {
    const float v2lo = v2 >= 0.f ? v2 * (1.f - kKeyTrunc) : v2 * (1.f + kKeyTrunc);
    const float xn = fmaxf(xnorm, 0.f);
    const float X = sqrtf(xn);
    const float cmax = __uint_as_float(*sb.cmax_bits);
    const float E = sb.ep * X * cmax + sb.en * (xn + cmax * cmax) + sb.ec * X * cmax;
    return v2lo - E + xn;
}

// Lloyd's bounds of a row for the next iteration, as distances: u >= the real
// distance to its center, l <= the real distance to every other center (FP32
// values carry at most W relative error; 1e-6 covers the rounding of these few
// operations).  l = 0: no bound.
__device__ __forceinline__ float bound_upper(float best, float W) { return sqrtf(best * (1.f + W)) * (1.f + 1e-6f); }
__device__ __forceinline__ float bound_lower(float l2, float xnorm, float W) {
    const float v = l2 * (1.f - 2.f * W) - 2.f * W * fmaxf(xnorm, 0.f);
    return v > 0.f ? sqrtf(v) * (1.f - 1e-6f) : 0.f;
}

// the distance that decides a row whose nearest screened center has exact FP32
// value b1 (FLT_MAX: none): see bound_certain
template <int MODE>
__device__ __forceinline__ float deciding(const float *D2, int64_t R, float b1) {
    return MODE == MODE_ROUND ? fminf(D2[R], b1) : b1;
}

// exact FP32 difference form of one row against one center, both in shared memory
// (8-byte loads when the row start is 8-byte aligned)
__device__ __forceinline__ float dist2_smem(const float *xa, const float *ca, int d, bool pairs) {
    float s = 0.f;
    if (pairs) {
        const float2 *x2 = reinterpret_cast<const float2 *>(xa);
        const float2 *c2 = reinterpret_cast<const float2 *>(ca);
#pragma unroll 4
        for (int p = 0; p < (d >> 1); ++p) {
            const float2 a = x2[p], c = c2[p];
            float t = __fsub_rn(a.x, c.x);
            s = __fmaf_rn(t, t, s);
            t = __fsub_rn(a.y, c.y);
            s = __fmaf_rn(t, t, s);
        }
        if (d & 1) {
            const float t = __fsub_rn(xa[d - 1], ca[d - 1]);
            s = __fmaf_rn(t, t, s);
        }
    } else {
#pragma unroll 4
        for (int q = 0; q < d; ++q) {
            const float t = __fsub_rn(xa[q], ca[q]);
            s = __fmaf_rn(t, t, s);
        }
    }
    return s;
}

// exact FP32 difference form of one row against several centers at once (rows in
// shared memory, 8-byte aligned): the chains are independent, so their FMA
// latencies overlap; each chain is still summed in ascending coordinates, so every
// value is bit-identical to dist2_fp32
template <int NC>
__device__ __forceinline__ void dist2_smem_multi(const float *xa, const float *const (&ca)[NC], int d, float (&s)[NC]) {
#pragma unroll
    for (int u = 0; u < NC; ++u) s[u] = 0.f;
    const float2 *x2 = reinterpret_cast<const float2 *>(xa);
#pragma unroll 2
    for (int p = 0; p < (d >> 1); ++p) {
        const float2 a = x2[p];
#pragma unroll
        for (int u = 0; u < NC; ++u) {
            const float2 c = reinterpret_cast<const float2 *>(ca[u])[p];
            float t = __fsub_rn(a.x, c.x);
            s[u] = __fmaf_rn(t, t, s[u]);
            t = __fsub_rn(a.y, c.y);
            s[u] = __fmaf_rn(t, t, s[u]);
        }
    }
    if (d & 1) {
#pragma unroll
        for (int u = 0; u < NC; ++u) {
            const float t = __fsub_rn(xa[d - 1], ca[u][d - 1]);
            s[u] = __fmaf_rn(t, t, s[u]);
        }
    }
}

// the pair's exact values in (value, center number) order; i2 = -1 when the pair
// has one real center
__device__ __forceinline__ void pair_top2(float va, int ja, float vb, int jb, bool has_b, float &b1, int &i1,
                                          float &b2, int &i2) {
    if (has_b && (vb < va || (vb == va && jb < ja))) { b1 = vb; i1 = jb; b2 = va; i2 = ja; }
    else { b1 = va; i1 = ja; b2 = has_b ? vb : FLT_MAX; i2 = has_b ? jb : -1; }
}

// Per-row copies: a warp takes 32 rows; asynchronous copies bring its 32 point
// rows and their pairs of center rows into shared memory (row stride = 2 mod 4:
// 8-byte aligned, conflict-free lane-per-row reads), then each lane sums its row.
template <int MODE>
__global__ void __launch_bounds__(256) refine_kernel(const float *__restrict__ X, int64_t n, int d,
                                                    const float *__restrict__ C, int c_cnt,
                                                    const int32_t *__restrict__ cand1, const float *__restrict__ v2s,
                                                    ScreenBound sb, float *D2, int32_t *idx, int32_t *labels,
                                                    const int32_t *prev, int *changed, float *dmin,
                                                    unsigned long long *fp64_cnt, unsigned long long *wide_cnt) {
    extern __shared__ __align__(16) float rsm[];
    const int ds = refine_stride(d);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float *xs = rsm + wid * 96 * ds;   // 32 point rows
    float *cs = xs + 32 * ds;          // 32 pairs of center rows
    const int64_t w0 = (int64_t)blockIdx.x * blockDim.x + wid * 32;
    const int nw = (int)max((int64_t)0, min((int64_t)32, n - w0));
    const int64_t R = w0 + lane;
    const int end = MODE == MODE_ROUND ? sb.st->batch_begin + sb.st->batch_cnt : c_cnt;
    int j = -1;
    if (lane < nw) j = cand1[R];
    const bool even = (d & 1) == 0;   // rows 8-byte aligned in global memory
    for (int rr = 0; rr < nw; ++rr) {
        const int jr = __shfl_sync(0xffffffffu, j, rr);
        if (jr < 0) continue;
        const int nc = jr + 1 < end ? 2 : 1;
        const float *xr = X + (w0 + rr) * d;
        const float *cr = C + (int64_t)jr * d;
        float *ct = cs + 2 * rr * ds;
        if (even) {
            for (int p = lane; p < (d >> 1); p += 32) {
                cp_async8(xs + rr * ds + 2 * p, xr + 2 * p);
                for (int u = 0; u < nc; ++u) cp_async8(ct + u * ds + 2 * p, cr + (int64_t)u * d + 2 * p);
            }
        } else {
            for (int q = lane; q < d; q += 32) {
                cp_async4(xs + rr * ds + q, xr + q);
                for (int u = 0; u < nc; ++u) cp_async4(ct + u * ds + q, cr + (int64_t)u * d + q);
            }
        }
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    bool fix = lane < nw && j < 0;
    int chg = 0;
    if (lane < nw && j >= 0) {
        const bool has_b = j + 1 < end;
        const float *ct = cs + 2 * lane * ds;
        const float *cp[2] = {ct, has_b ? ct + ds : ct};
        float v[2];
        dist2_smem_multi<2>(xs + lane * ds, cp, d, v);
        const float va = v[0], vb = has_b ? v[1] : 0.f;
        float b1, b2;
        int i1, i2;
        pair_top2(va, j, vb, j + 1, has_b, b1, i1, b2, i2);
        const float m = deciding<MODE>(D2, R, b1);
        if (pair_certain(sb, sb.xnorm[R], m, v2s[R], d))
            chg = decide_top2<MODE>(X, d, C, R, b1, i1, b2, i2, D2, idx, labels, prev, dmin, fp64_cnt, wide_cnt);
        else {
            fix = true;
            sb.ub[R] = m;
        }
    } else if (fix) {
        sb.ub[R] = deciding<MODE>(D2, R, FLT_MAX);
    }
    append_fixups(sb, fix, R);
    if (MODE == MODE_ASSIGN && changed) {
        const int c = warp_sum_i32(chg);
        if (lane == 0 && c) atomicAdd(changed, c);
    }
}

// Per-row refine for rows of d = 0 mod 4 floats (16-byte aligned): one thread per
// row sums every center of its screened group (G adjacent centers) with G
// interleaved exact FP32 chains (ascending coordinates, bit-identical to
// dist2_fp32) from 16-byte loads of the point row and the center rows; no
// shared-memory staging, so the kernel runs at full occupancy and the rows come
// through L1.  The lexicographic top-2 of the group then goes through the same
// certainty test and decision as a pair.
template <int MODE, int G>
__global__ void __launch_bounds__(256) refine_direct_kernel(const float *__restrict__ X, int64_t n, int d,
                                                           const float *__restrict__ C, int c_cnt,
                                                           const int32_t *__restrict__ cand1,
                                                           const float *__restrict__ v2s, ScreenBound sb, float *D2,
                                                           int32_t *idx, int32_t *labels, const int32_t *prev,
                                                           int *changed, float *dmin, unsigned long long *fp64_cnt,
                                                           unsigned long long *wide_cnt, const int32_t *order,
                                                           const int *nrows_dev, float *ubd, float *lbd) {
    // rows in the order given (a permutation of 0..n-1, e.g. the rows sorted by
    // their previous label: neighbouring threads then mostly read the same center
    // rows, which L1 serves), or in storage order.  nrows_dev: a compact pass over
    // the rows order[0 .. *nrows_dev), whose screening results are by position.
    const int64_t T = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = T < (nrows_dev ? (int64_t)*nrows_dev : n);
    const int64_t R = order && valid ? (int64_t)order[T] : T;
    const int64_t Ri = nrows_dev ? T : R;
    const int lane = threadIdx.x & 31;
    const int end = MODE == MODE_ROUND ? sb.st->batch_begin + sb.st->batch_cnt : c_cnt;
    const int j = valid ? cand1[Ri] : -1;
    if (MODE == MODE_ASSIGN && lbd && valid) lbd[R] = 0.f;   // no bound unless the row is certified below
    bool fix = valid && j < 0;
    int chg = 0;
    if (valid && j >= 0) {
        const float4 *x4 = reinterpret_cast<const float4 *>(X + R * d);
        const float4 *c4[G];
#pragma unroll
        for (int u = 0; u < G; ++u) c4[u] = reinterpret_cast<const float4 *>(C + (int64_t)min(j + u, end - 1) * d);
        float v[G];
#pragma unroll
        for (int u = 0; u < G; ++u) v[u] = 0.f;
#pragma unroll 2
        for (int p = 0; p < (d >> 2); ++p) {
            const float4 x = __ldg(x4 + p);
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const float4 c = __ldg(c4[u] + p);
                float t;
                t = __fsub_rn(x.x, c.x); v[u] = __fmaf_rn(t, t, v[u]);
                t = __fsub_rn(x.y, c.y); v[u] = __fmaf_rn(t, t, v[u]);
                t = __fsub_rn(x.z, c.z); v[u] = __fmaf_rn(t, t, v[u]);
                t = __fsub_rn(x.w, c.w); v[u] = __fmaf_rn(t, t, v[u]);
            }
        }
        // lexicographic (value, center number) top-2 over the group's real centers
        float b1 = FLT_MAX, b2 = FLT_MAX;
        int i1 = INT_MAX, i2 = -1;
#pragma unroll
        for (int u = 0; u < G; ++u) {
            if (j + u < end) {
                if (v[u] < b1) { b2 = b1; i2 = i1 == INT_MAX ? -1 : i1; b1 = v[u]; i1 = j + u; }
                else if (v[u] < b2) { b2 = v[u]; i2 = j + u; }
            }
        }
        if (i2 < 0) b2 = FLT_MAX;
        const float m = deciding<MODE>(D2, R, b1);
        const float v2r = v2s[Ri];
        if (pair_certain(sb, sb.xnorm[R], m, v2r, d)) {
            chg = decide_top2<MODE>(X, d, C, R, b1, i1, b2, i2, D2, idx, labels, prev, dmin, fp64_cnt, wide_cnt);
            if (MODE == MODE_ASSIGN && lbd) {
                // the group's runner-up (exact FP32) and the bound outside the group
                const float W = fp32_tie_window(d);
                const bool first = labels[R] == i1;
                const float runner = first ? b2 : b1;
                ubd[R] = bound_upper(first ? b1 : b2, W);
                lbd[R] = bound_lower(fminf(runner, outside_lb(sb, sb.xnorm[R], v2r)), sb.xnorm[R], W);
            }
        } else {
            fix = true;
            sb.ub[R] = m;
        }
    } else if (fix) {
        sb.ub[R] = deciding<MODE>(D2, R, FLT_MAX);
    }
    append_fixups(sb, fix, R);
    if (MODE == MODE_ASSIGN && changed) {
        const int c = warp_sum_i32(chg);
        if (lane == 0 && c) atomicAdd(changed, c);
    }
}

// Centers resident in shared memory (used when lane-per-row reads are conflict-free:
// d odd or d = 2 mod 4).  Persistent CTAs copy the pass's centers once; each warp
// then walks 32-row blocks of X.  A block is contiguous in X, so flat 16-byte
// asynchronous copies bring it in, double-buffered per warp, and the next block's
// screening results are loaded while the current block is summed.  A pass whose
// centers exceed shared memory runs as a few launches, each holding the slice
// [part_lo, part_lo + part_rows) of the centers (plus the next row, the partner of
// a pair that ends the slice): a row is refined by the launch whose slice holds its
// screened pair, and rows without one are listed for the fix-up by the first.
__host__ __device__ __forceinline__ int resident_center_floats(int cap_rows, int d) { return (cap_rows * d + 3) & ~3; }
__host__ __device__ __forceinline__ int resident_block_floats(int d) { return (32 * d + 3) & ~3; }

template <int MODE>
__global__ void __launch_bounds__(512) refine_resident_kernel(
    const float *__restrict__ X, int64_t n, int d, const float *__restrict__ C, int cap_rows, int part_lo,
    int part_rows, int hold_rows, const int32_t *__restrict__ cand1, const float *__restrict__ v2s, ScreenBound sb,
    float *D2, int32_t *idx, int32_t *labels, const int32_t *prev, int *changed, float *dmin,
    unsigned long long *fp64_cnt, unsigned long long *wide_cnt) {
    extern __shared__ __align__(16) float rsm[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int begin = MODE == MODE_ROUND ? sb.st->batch_begin : 0;
    const int cnt = MODE == MODE_ROUND ? min(sb.st->batch_cnt, cap_rows) : cap_rows;
    const int lo = part_lo, hi = min(cnt, part_lo + part_rows);
    if (lo > 0 && lo >= hi) return;   // uniform per block: the batch ends before this slice
    const int nhold = max(0, min(cnt, hi + 1) - lo);   // <= hold_rows
    const int xfl = resident_block_floats(d);
    float *Cs = rsm;
    float *xb = rsm + resident_center_floats(hold_rows, d) + wid * 2 * xfl;
    {
        const float *src = C + (int64_t)(begin + lo) * d;
        const int nf = nhold * d;
        if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
            for (int f = threadIdx.x; f < (nf >> 2); f += blockDim.x) cp_async16(Cs + 4 * f, src + 4 * f);
            for (int f = (nf & ~3) + threadIdx.x; f < nf; f += blockDim.x) cp_async4(Cs + f, src + f);
        } else {
            for (int f = threadIdx.x; f < nf; f += blockDim.x) cp_async4(Cs + f, src + f);
        }
        cp_async_commit();
    }
    const int64_t nb = (n + 31) / 32;
    const int64_t gw = (int64_t)blockIdx.x * nwarps + wid, W = (int64_t)gridDim.x * nwarps;
    // a block starts at 32 b d floats = 128 b d bytes: 16-byte aligned when X is
    const bool xal = (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
    auto issue = [&](int64_t b, float *dst) {
        const int64_t r0 = b * 32;
        const int nf = (int)min((int64_t)32, n - r0) * d;
        const float *src = X + r0 * d;
        if (xal) {
            for (int f = lane; f < (nf >> 2); f += 32) cp_async16(dst + 4 * f, src + 4 * f);
            for (int f = (nf & ~3) + lane; f < nf; f += 32) cp_async4(dst + f, src + f);
        } else {
            for (int f = lane; f < nf; f += 32) cp_async4(dst + f, src + f);
        }
    };
    // screening results of block b for this lane's row
    auto fetch = [&](int64_t b, int &j, float &v2, float &xn) {
        const int64_t R = b * 32 + lane;
        j = -1;
        v2 = 0.f;
        xn = 0.f;
        if (b < nb && R < n) {
            j = cand1[R];
            v2 = v2s[R];
            xn = sb.xnorm[R];
        }
    };
    if (gw < nb) issue(gw, xb);
    cp_async_commit();
    int jn;
    float v2n, xnn;
    fetch(gw, jn, v2n, xnn);
    cp_async_wait<1>();   // the centers (the first block may still be in flight)
    __syncthreads();
    const bool pairs = (d & 1) == 0;
    int chg = 0, it = 0;
    for (int64_t b = gw; b < nb; b += W, ++it) {
        const float *cur = xb + (it & 1) * xfl;
        if (b + W < nb) issue(b + W, xb + ((it + 1) & 1) * xfl);
        cp_async_commit();
        int j = jn;
        const float v2 = v2n, xn = xnn;
        fetch(b + W, jn, v2n, xnn);
        const int64_t R = b * 32 + lane;
        const bool valid = R < n;
        cp_async_wait<1>();   // this block is in (the next one may be pending)
        __syncwarp();
        const int jl = j - begin;   // batch-local pair start (j = -1: none)
        const bool screened = j >= 0 && jl >= 0 && jl < cnt;
        bool fix = valid && !screened && lo == 0;
        if (valid && screened && jl >= lo && jl < hi) {
            const bool has_b = jl + 1 < cnt;
            const float *xa = cur + lane * d;
            const float *ca = Cs + (int64_t)(jl - lo) * d;
            float va, vb = 0.f;
            if (pairs) {
                const float *cp[2] = {ca, has_b ? ca + d : ca};
                float v[2];
                dist2_smem_multi<2>(xa, cp, d, v);
                va = v[0];
                if (has_b) vb = v[1];
            } else {
                va = dist2_smem(xa, ca, d, false);
                if (has_b) vb = dist2_smem(xa, ca + d, d, false);
            }
            float b1, b2;
            int i1, i2;
            pair_top2(va, j, vb, j + 1, has_b, b1, i1, b2, i2);
            const float m = deciding<MODE>(D2, R, b1);
            if (pair_certain(sb, xn, m, v2, d))
                chg += decide_top2<MODE>(X, d, C, R, b1, i1, b2, i2, D2, idx, labels, prev, dmin, fp64_cnt, wide_cnt);
            else {
                fix = true;
                sb.ub[R] = m;
            }
        } else if (fix) {
            sb.ub[R] = deciding<MODE>(D2, R, FLT_MAX);
        }
        append_fixups(sb, fix, R);
        __syncwarp();   // the buffer is refilled two blocks later
    }
    cp_async_wait<0>();
    if (MODE == MODE_ASSIGN && changed) {
        const int c = warp_sum_i32(chg);
        if (lane == 0 && c) atomicAdd(changed, c);
    }
}

// warps of a resident refine CTA holding all cap_rows centers (0: they do not fit,
// or the stride is not conflict-free)
int resident_warps(int cap_rows, int d) {
    if (!((d & 1) || (d & 3) == 2)) return 0;
    const size_t budget = 200u * 1024u;
    const size_t cbytes = sizeof(float) * (size_t)resident_center_floats(cap_rows, d);
    if (cbytes >= budget) return 0;
    const size_t per_warp = sizeof(float) * 2 * (size_t)resident_block_floats(d);
    const int w = (int)((budget - cbytes) / per_warp);
    return w < 4 ? 0 : (w > 16 ? 16 : w);
}

size_t resident_smem_bytes(int cap_rows, int d, int warps) {
    return sizeof(float) * ((size_t)resident_center_floats(cap_rows, d) + (size_t)warps * 2 * resident_block_floats(d));
}

// How the resident refine covers a pass of cap_rows centers: `parts` launches of
// `rows` centers each (`hold` rows of shared memory, `warps` warps per CTA).
// parts = 0: the per-row kernel (refine_kernel) is used instead.
struct ResidentPlan {
    int parts, rows, hold, warps;
};

ResidentPlan resident_plan(int cap_rows, int d) {
    const int w1 = resident_warps(cap_rows, d);
    if (w1 > 0) return {1, cap_rows, cap_rows, w1};
    if (!((d & 1) || (d & 3) == 2)) return {0, 0, 0, 0};
    // slices: 8 warps, the rest of the 200 KB for one slice of centers plus the
    // partner row; each launch reads X once, so at most 3 of them
    const int warps = 8;
    const size_t per_warp = sizeof(float) * 2 * (size_t)resident_block_floats(d);
    if (warps * per_warp + sizeof(float) * 66 * (size_t)d + 16 > 200u * 1024u) return {0, 0, 0, 0};
    const size_t cfloats = (200u * 1024u - warps * per_warp) / sizeof(float);
    const int hold = (int)((cfloats - 3) / (size_t)d);   // resident_center_floats adds at most 3
    const int rows = (hold - 1) & ~1;
    if (rows < 64) return {0, 0, 0, 0};
    const int parts = (cap_rows + rows - 1) / rows;
    if (parts > 3) return {0, 0, 0, 0};
    return {parts, rows, rows + 1, warps};
}

// warps per refine CTA: 96 staged rows (32 points, 32 pairs of centers) of
// refine_stride(d) floats each, within 200 KB
int refine_warps(int d) {
    const int w = (int)((200u * 1024u) / (96u * 4u * (unsigned)refine_stride(d)));
    return w > 8 ? 8 : (w < 1 ? 1 : w);
}

size_t refine_smem_bytes(int d) { return sizeof(float) * refine_warps(d) * 96 * (size_t)refine_stride(d); }

// Rows the screening could not settle, scanned exactly against every center of the
// pass.  A CTA takes tiles of 32 listed rows, four per warp; the centers stream
// through shared memory in chunks of 64 (asynchronous copies, double-buffered) and
// lane l sums centers l and l + 32 of each chunk for the warp's four rows in the
// exact FP32 difference form in ascending coordinates (bit-identical to
// dist2_fp32): per coordinate pair four broadcast and two conflict-free 8-byte
// shared loads (row stride 2 mod 4) feed 32 FP32 operations, and every center chunk
// serves 32 rows.  A lexicographic top-2 per row is merged across the warp, then the
// same decision as nearest_kernel (decide_top2).  Persistent: the row count is read
// on the device.
constexpr int kFxWarpRows = 4;
constexpr int kFxRows = 8 * kFxWarpRows;
constexpr int kFxCent = 64;

template <int MODE>
__global__ void __launch_bounds__(256) fixup_kernel(const float *__restrict__ X, int d, const float *__restrict__ C,
                                                   int c_cnt, int c_pairs, const DevState *st,
                                                   const int32_t *__restrict__ rows, const int *rows_cnt, float *D2,
                                                   int32_t *idx, int32_t *labels, const int32_t *prev, int *changed,
                                                   float *dmin, unsigned long long *fp64_cnt,
                                                   unsigned long long *wide_cnt) {
    extern __shared__ __align__(16) float fsm[];
    const int ds = refine_stride(d);
    float *xs = fsm;                   // kFxRows x ds point rows (row wid + 8 r of the tile: xs + (wid + 8 r) ds)
    float *cs = fsm + kFxRows * ds;    // 2 x kFxCent x ds center rows
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nrows = *rows_cnt;
    const int begin = MODE == MODE_ROUND ? st->batch_begin : 0;
    const int cnt = MODE == MODE_ROUND ? st->batch_cnt : c_cnt;
    const int nchunk = (cnt + kFxCent - 1) / kFxCent;
    const float FMAX = FLT_MAX;
    auto issue = [&](int ch) {
        float *dst = cs + (ch & 1) * kFxCent * ds;
        const int j0 = ch * kFxCent;
        const int nc = min(kFxCent, cnt - j0);
        for (int rr = wid; rr < nc; rr += 8) {
            const float *src = C + (int64_t)(begin + j0 + rr) * d;
            if (c_pairs)
                for (int p = lane; p < (d >> 1); p += 32) cp_async8(dst + rr * ds + 2 * p, src + 2 * p);
            for (int q = (c_pairs ? (d & ~1) : 0) + lane; q < d; q += 32) cp_async4(dst + rr * ds + q, src + q);
        }
    };
    for (int t0 = blockIdx.x * kFxRows; t0 < nrows; t0 += gridDim.x * kFxRows) {   // uniform per block
        const int nr = min(kFxRows, nrows - t0);
        __syncthreads();   // the previous tile's readers are done with xs and cs
#pragma unroll
        for (int r = 0; r < kFxWarpRows; ++r) {
            const int tr = wid + 8 * r;
            if (tr < nr) {
                const float *src = X + (int64_t)rows[t0 + tr] * d;
                for (int q = lane; q < d; q += 32) xs[tr * ds + q] = __ldg(src + q);
            }
        }
        if (nchunk > 0) issue(0);
        cp_async_commit();
        float b1[kFxWarpRows], b2[kFxWarpRows];
        int i1[kFxWarpRows], i2[kFxWarpRows];
#pragma unroll
        for (int r = 0; r < kFxWarpRows; ++r) { b1[r] = FMAX; b2[r] = FMAX; i1[r] = INT_MAX; i2[r] = INT_MAX; }
        for (int ch = 0; ch < nchunk; ++ch) {
            if (ch + 1 < nchunk) issue(ch + 1);
            cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();   // chunk ch and the point rows are visible
            const float *cb = cs + (ch & 1) * kFxCent * ds;
            const float *c0 = cb + lane * ds, *c1 = cb + (lane + 32) * ds;
            float a0[kFxWarpRows], a1[kFxWarpRows];
#pragma unroll
            for (int r = 0; r < kFxWarpRows; ++r) { a0[r] = 0.f; a1[r] = 0.f; }
            const float2 *p0 = reinterpret_cast<const float2 *>(c0);
            const float2 *p1 = reinterpret_cast<const float2 *>(c1);
#pragma unroll 2
            for (int p = 0; p < (d >> 1); ++p) {
                const float2 u = p0[p], v = p1[p];
#pragma unroll
                for (int r = 0; r < kFxWarpRows; ++r) {
                    const float2 x = reinterpret_cast<const float2 *>(xs + (wid + 8 * r) * ds)[p];
                    float t = __fsub_rn(x.x, u.x);
                    a0[r] = __fmaf_rn(t, t, a0[r]);
                    t = __fsub_rn(x.y, u.y);
                    a0[r] = __fmaf_rn(t, t, a0[r]);
                    t = __fsub_rn(x.x, v.x);
                    a1[r] = __fmaf_rn(t, t, a1[r]);
                    t = __fsub_rn(x.y, v.y);
                    a1[r] = __fmaf_rn(t, t, a1[r]);
                }
            }
            if (d & 1) {
#pragma unroll
                for (int r = 0; r < kFxWarpRows; ++r) {
                    const float xe = xs[(wid + 8 * r) * ds + d - 1];
                    float t = __fsub_rn(xe, c0[d - 1]);
                    a0[r] = __fmaf_rn(t, t, a0[r]);
                    t = __fsub_rn(xe, c1[d - 1]);
                    a1[r] = __fmaf_rn(t, t, a1[r]);
                }
            }
            const int jl0 = ch * kFxCent + lane, jl1 = jl0 + 32;
#pragma unroll
            for (int r = 0; r < kFxWarpRows; ++r) {
                if (jl0 < cnt && lex_lt(a0[r], begin + jl0, b2[r], i2[r])) {
                    if (lex_lt(a0[r], begin + jl0, b1[r], i1[r])) {
                        b2[r] = b1[r]; i2[r] = i1[r]; b1[r] = a0[r]; i1[r] = begin + jl0;
                    } else {
                        b2[r] = a0[r]; i2[r] = begin + jl0;
                    }
                }
                if (jl1 < cnt && lex_lt(a1[r], begin + jl1, b2[r], i2[r])) {
                    if (lex_lt(a1[r], begin + jl1, b1[r], i1[r])) {
                        b2[r] = b1[r]; i2[r] = i1[r]; b1[r] = a1[r]; i1[r] = begin + jl1;
                    } else {
                        b2[r] = a1[r]; i2[r] = begin + jl1;
                    }
                }
            }
            __syncthreads();   // every reader is done with this buffer before it is refilled
        }
        cp_async_wait<0>();
#pragma unroll
        for (int r = 0; r < kFxWarpRows; ++r) {
            float v1 = b1[r], v2 = b2[r];
            int j1 = i1[r], j2 = i2[r];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float c1v = __shfl_xor_sync(0xffffffffu, v1, o), c2v = __shfl_xor_sync(0xffffffffu, v2, o);
                const int k1 = __shfl_xor_sync(0xffffffffu, j1, o), k2 = __shfl_xor_sync(0xffffffffu, j2, o);
                top2_merge(v1, j1, v2, j2, c1v, k1, c2v, k2);
            }
            const int tr = wid + 8 * r;
            if (lane == 0 && tr < nr) {
                const int64_t R = rows[t0 + tr];
                if (j2 == INT_MAX) { j2 = -1; v2 = FMAX; }
                if (decide_top2<MODE>(X, d, C, R, v1, j1, v2, j2, D2, idx, labels, prev, dmin, fp64_cnt, wide_cnt) &&
                    changed)
                    atomicAdd(changed, 1);
            }
        }
    }
}

// Fix-up with the pass's centers resident in shared memory (used when they fit):
// persistent CTAs copy the centers once (row stride 2 mod 4: lane l reading center
// l of a consecutive run is conflict-free with 8-byte loads); then one warp per
// listed row: the row is staged, lane l sums centers l, l + 32, ... in the exact
// FP32 difference form (bit-identical to dist2_fp32), a lexicographic top-2 is
// merged across the warp and decided by decide_top2.  No center is read from
// global memory more than once per CTA.  Listed row t goes to CTA t mod G (G CTAs),
// so when the rows outnumber the warps the warps that take a second row are spread
// one or two per SM instead of filling the first SMs.
template <int MODE>
__global__ void __launch_bounds__(512) fixup_resident_kernel(const float *__restrict__ X, int d,
                                                            const float *__restrict__ C, int c_cnt, int cap_rows,
                                                            int c_pairs, const DevState *st,
                                                            const int32_t *__restrict__ rows, const int *rows_cnt,
                                                            float *D2, int32_t *idx, int32_t *labels,
                                                            const int32_t *prev, int *changed, float *dmin,
                                                            unsigned long long *fp64_cnt,
                                                            unsigned long long *wide_cnt) {
    extern __shared__ __align__(16) float fsm[];
    const int ds = refine_stride(d);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nrows = *rows_cnt;
    if ((int)blockIdx.x >= nrows) return;   // uniform per block: nothing for this CTA
    const int begin = MODE == MODE_ROUND ? st->batch_begin : 0;
    const int cnt = MODE == MODE_ROUND ? min(st->batch_cnt, cap_rows) : c_cnt;
    float *Cs = fsm;                                   // cap_rows x ds
    float *xs = fsm + (size_t)cap_rows * ds + wid * ds; // this warp's point row
    for (int rr = wid; rr < cnt; rr += nwarps) {
        const float *src = C + (int64_t)(begin + rr) * d;
        if (c_pairs)
            for (int p = lane; p < (d >> 1); p += 32) cp_async8(Cs + rr * ds + 2 * p, src + 2 * p);
        for (int q = (c_pairs ? (d & ~1) : 0) + lane; q < d; q += 32) cp_async4(Cs + rr * ds + q, src + q);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const float FMAX = FLT_MAX;
    for (int t = wid * gridDim.x + blockIdx.x; t < nrows; t += gridDim.x * nwarps) {   // uniform per warp
        const int64_t R = rows[t];
        for (int q = lane; q < d; q += 32) xs[q] = __ldg(X + R * d + q);
        __syncwarp();
        float b1 = FMAX, b2 = FMAX;
        int i1 = INT_MAX, i2 = INT_MAX;
        // lane l: centers l, l + 32, l + 64, l + 96 summed together, then the next 128
        for (int j0 = lane; j0 < cnt; j0 += 128) {
            const float *cp[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) cp[u] = Cs + (size_t)min(j0 + 32 * u, cnt - 1) * ds;
            float v[4];
            dist2_smem_multi<4>(xs, cp, d, v);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int jl = j0 + 32 * u;
                if (jl < cnt) {
                    const int j = begin + jl;
                    if (lex_lt(v[u], j, b2, i2)) {
                        if (lex_lt(v[u], j, b1, i1)) { b2 = b1; i2 = i1; b1 = v[u]; i1 = j; }
                        else { b2 = v[u]; i2 = j; }
                    }
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float c1 = __shfl_xor_sync(0xffffffffu, b1, o), c2 = __shfl_xor_sync(0xffffffffu, b2, o);
            const int j1 = __shfl_xor_sync(0xffffffffu, i1, o), j2 = __shfl_xor_sync(0xffffffffu, i2, o);
            top2_merge(b1, i1, b2, i2, c1, j1, c2, j2);
        }
        if (lane == 0) {
            if (i2 == INT_MAX) { i2 = -1; b2 = FMAX; }
            if (decide_top2<MODE>(X, d, C, R, b1, i1, b2, i2, D2, idx, labels, prev, dmin, fp64_cnt, wide_cnt) &&
                changed)
                atomicAdd(changed, 1);
        }
        __syncwarp();   // the staged row is read before the next one overwrites it
    }
}

// warps of a resident fix-up CTA (0: the centers do not fit; use fixup_kernel)
int fixup_resident_warps(int cap_rows, int d) {
    const size_t budget = 200u * 1024u;
    const size_t cbytes = sizeof(float) * (size_t)cap_rows * refine_stride(d);
    const size_t per_warp = sizeof(float) * (size_t)refine_stride(d);
    if (cbytes + 16 * per_warp > budget) return 0;
    return 16;
}

size_t fixup_smem_bytes(int d) { return sizeof(float) * (size_t)(kFxRows + 2 * kFxCent) * refine_stride(d); }

cudaError_t launch_fixup(const Ctx &c, int mode_round, const float *C, int k, int32_t *labels, const int32_t *prev,
                         int *changed, float *dmin, const int32_t *rows, const int *rows_cnt) {
    // 8-byte center copies need d even and 8-byte aligned rows
    const int c_pairs = (c.d % 2 == 0) && (reinterpret_cast<uintptr_t>(C) % 8 == 0);
    const int cap_rows = mode_round ? c.cap_round : k;
    const int rw = fixup_resident_warps(cap_rows, c.d);
    if (rw > 0) {
        const size_t sm = sizeof(float) * ((size_t)cap_rows + rw) * refine_stride(c.d);
        if (mode_round)
            fixup_resident_kernel<MODE_ROUND><<<c.num_sms, 32 * rw, sm, c.stream>>>(
                c.X, c.d, C, 0, cap_rows, c_pairs, c.st, rows, rows_cnt, c.D2, c.idx, nullptr, nullptr,
                nullptr, nullptr, &c.st->argmin_fp64, &c.st->argmin_wide);
        else
            fixup_resident_kernel<MODE_ASSIGN><<<c.num_sms, 32 * rw, sm, c.stream>>>(
                c.X, c.d, C, k, cap_rows, c_pairs, c.st, rows, rows_cnt, nullptr, nullptr, labels, prev,
                changed, dmin, &c.st->argmin_fp64, &c.st->argmin_wide);
        count_launches(1);
        return cudaGetLastError();
    }
    const int grid = c.num_sms * 4;   // persistent: the row count is only known on the device
    const size_t sm = fixup_smem_bytes(c.d);
    const int pairs = c_pairs;
    if (mode_round)
        fixup_kernel<MODE_ROUND><<<grid, 256, sm, c.stream>>>(c.X, c.d, C, 0, pairs, c.st, rows, rows_cnt, c.D2,
                                                              c.idx, nullptr, nullptr, nullptr, nullptr,
                                                              &c.st->argmin_fp64, &c.st->argmin_wide);
    else
        fixup_kernel<MODE_ASSIGN><<<grid, 256, sm, c.stream>>>(c.X, c.d, C, k, pairs, c.st, rows, rows_cnt,
                                                               nullptr, nullptr, labels, prev, changed, dmin,
                                                               &c.st->argmin_fp64, &c.st->argmin_wide);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t configure_refine_kernels() {
    // the tensor passes support d + 2 <= 192: refine tiles of 256 rows of up to 190 floats
    cudaError_t e = cudaFuncSetAttribute(refine_kernel<MODE_ROUND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(refine_kernel<MODE_ASSIGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(refine_resident_kernel<MODE_ROUND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(refine_resident_kernel<MODE_ASSIGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
    if (e != cudaSuccess) return e;
    // the tensor passes support d <= 190: fix-up tiles of 160 rows of up to 190 floats
    const int fx = (int)fixup_smem_bytes(190);
    e = cudaFuncSetAttribute(fixup_kernel<MODE_ROUND>, cudaFuncAttributeMaxDynamicSharedMemorySize, fx);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fixup_kernel<MODE_ASSIGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, fx);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fixup_resident_kernel<MODE_ROUND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fixup_resident_kernel<MODE_ASSIGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024);
}

// exact FP32 difference form of one row against one center, both in global memory:
// the same chain as dist2_fp32 (ascending coordinates, one rounded subtraction and
// one FMA each), with 16-byte loads when both rows are 16-byte aligned
__device__ __forceinline__ float dist2_fp32_v4(const float *__restrict__ x, const float *__restrict__ c, int d) {
    if ((d & 3) == 0 && ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(c)) & 15u) == 0) {
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        const float4 *c4 = reinterpret_cast<const float4 *>(c);
        float s = 0.f;
        for (int p = 0; p < (d >> 2); ++p) {
            const float4 a = __ldg(x4 + p), b = __ldg(c4 + p);
            float t = __fsub_rn(a.x, b.x);
            s = __fmaf_rn(t, t, s);
            t = __fsub_rn(a.y, b.y);
            s = __fmaf_rn(t, t, s);
            t = __fsub_rn(a.z, b.z);
            s = __fmaf_rn(t, t, s);
            t = __fsub_rn(a.w, b.w);
            s = __fmaf_rn(t, t, s);
        }
        return s;
    }
    return dist2_fp32(x, c, d);
}

// Rows the list pass screened (rows[i], i < *rows_cnt): one warp per row.  The
// row's four column groups listed their centers whose screened value is at most
// thr[i]; lane l computes listed center l in the exact FP32 difference form
// (bit-identical to dist2_fp32), a lexicographic top-2 is merged across the warp,
// and the row is certain when no group overflowed its slots and every center
// left off the list (screened value above thr[i]) is, by the screening bound,
// beyond the tie window of the deciding distance (bound_certain).  Certain rows
// take decide_top2, the others go to the exact scan's list (rows2).
template <int MODE, bool BYROW>
__global__ void __launch_bounds__(256) refine_list_kernel(
    const float *__restrict__ X, int d, const float *__restrict__ C, int c_cnt, const int32_t *__restrict__ rows,
    const int *rows_cnt, const int32_t *__restrict__ lst, const int32_t *__restrict__ lcnt,
    const float *__restrict__ thr, ScreenBound sb, int32_t *rows2, int *cnt2, float *D2, int32_t *idx,
    int32_t *labels, const int32_t *prev, int *changed, float *dmin, unsigned long long *fp64_cnt,
    unsigned long long *wide_cnt) {
    // four listed rows per warp, eight lanes per row (a row's lists usually hold a
    // few centers): lane sl of a row's group takes its list entries sl, sl + 8, ...
    constexpr int S = tc::kListSlots;
    const int lane = threadIdx.x & 31;
    const int sub = lane >> 3, sl = lane & 7;
    const unsigned gmask = 0xFFu << (8 * sub);   // the lanes of this row's group
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nrows = *rows_cnt;
    const int begin = MODE == MODE_ROUND ? sb.st->batch_begin : 0;
    const int cnt = MODE == MODE_ROUND ? sb.st->batch_cnt : c_cnt;
    const float FMAX = FLT_MAX;
    for (int64_t i0 = gw * 4; i0 < nrows; i0 += W * 4) {   // uniform per warp
        const int64_t i = i0 + sub;
        const bool valid = i < nrows;
        const int64_t R = valid ? rows[i] : 0;
        const int64_t li = BYROW ? R : i;   // the row's lists and threshold: by row, or by list position
        const int cg = valid && sl < 4 ? lcnt[li * 4 + sl] : 0;
        const bool over = (__ballot_sync(0xffffffffu, cg > S) & gmask) != 0;
        const int c0 = __shfl_sync(0xffffffffu, cg, 8 * sub), c1 = __shfl_sync(0xffffffffu, cg, 8 * sub + 1);
        const int c2 = __shfl_sync(0xffffffffu, cg, 8 * sub + 2), c3 = __shfl_sync(0xffffffffu, cg, 8 * sub + 3);
        float b1 = FMAX, b2 = FMAX;
        int i1 = INT_MAX, i2 = INT_MAX;
        if (valid && !over) {
            const int total = c0 + c1 + c2 + c3;
            for (int e = sl; e < total; e += 8) {
                int g, sidx = e;
                if (sidx < c0) g = 0;
                else if ((sidx -= c0) < c1) g = 1;
                else if ((sidx -= c1) < c2) g = 2;
                else { sidx -= c2; g = 3; }
                const int col = lst[(li * 4 + g) * S + sidx];
                if (col >= 0 && col < cnt) {
                    const int j = begin + col;
                    const float v = dist2_fp32_v4(X + R * d, C + (int64_t)j * d, d);
                    if (lex_lt(v, j, b2, i2)) {
                        if (lex_lt(v, j, b1, i1)) { b2 = b1; i2 = i1; b1 = v; i1 = j; }
                        else { b2 = v; i2 = j; }
                    }
                }
            }
        }
        // top-2 of the row's group (xor offsets below 8 stay within the group)
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            const float u1 = __shfl_xor_sync(0xffffffffu, b1, o), u2 = __shfl_xor_sync(0xffffffffu, b2, o);
            const int j1 = __shfl_xor_sync(0xffffffffu, i1, o), j2 = __shfl_xor_sync(0xffffffffu, i2, o);
            top2_merge(b1, i1, b2, i2, u1, j1, u2, j2);
        }
        if (sl == 0 && valid) {
            bool certain = false;
            if (!over) {
                const float m = deciding<MODE>(D2, R, i1 != INT_MAX ? b1 : FMAX);
                certain = m < FMAX && bound_certain(sb, sb.xnorm[R], m, thr[li], d);
            }
            if (certain) {
                if (i2 == INT_MAX) { i2 = -1; b2 = FMAX; }
                if (decide_top2<MODE>(X, d, C, R, b1, i1, b2, i2, D2, idx, labels, prev, dmin, fp64_cnt, wide_cnt) &&
                    changed)
                    atomicAdd(changed, 1);
            } else {
                rows2[atomicAdd(cnt2, 1)] = (int32_t)R;
            }
        }
    }
}

// A distance pass on the tensor cores.  rows / rows_cnt (Lloyd, direct refine
// only): the pass covers just the rows rows[0 .. *rows_cnt), gathered into a compact
// image; the others keep what the caller wrote for them.
cudaError_t launch_tc_pass(Ctx &c, int mode_round, const float *C, int k, int32_t *labels, const int32_t *prev,
                           int *changed, float *dmin, int timing_cls, const int32_t *rows, const int *rows_cnt) {
    cudaError_t e;
    const int fmt = c.tc_fmt;
    if ((e = tc::launch_prep_centers(C, c.d, fmt, c.st, k, mode_round, mode_round ? c.cap_round : k, c.tc_anchor,
                                     c.tc_img, c.tc_ncol, c.tc_tscale, c.tc_cmax, c.stream)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(c.fix_cnt, 0, sizeof(int), c.stream)) != cudaSuccess) return e;
    // rows the screening does not reach (e.g. an empty batch) must not see a stale winner
    if (!rows && (e = cudaMemsetAsync(c.cand1, 0xFF, sizeof(int32_t) * (size_t)c.n, c.stream)) != cudaSuccess)
        return e;
    tc::TcParams p{};
    p.X = c.X; p.n = c.n; p.d = c.d; p.fmt = fmt;
    p.ximg = c.tc_ximg; p.xnorm = c.tc_xnorm; p.xscale = c.tc_xscale;
    p.Cf = C; p.cnt = k; p.st = c.st; p.bimg = c.tc_img; p.ncol = c.tc_ncol; p.tscale = c.tc_tscale;
    p.cmax_bits = c.tc_cmax;
    p.cand1 = c.cand1; p.v2 = c.tc_v2; p.fix_rows = c.fix_rows; p.fix_cnt = c.fix_cnt;
    p.fp64_cnt = &c.st->argmin_fp64; p.err = c.tc_err;
    const int cap_rows = mode_round ? c.cap_round : k;
    const ResidentPlan rp = resident_plan(cap_rows, c.d);
    // the direct refine serves rows of d = 0 mod 4; with it, formats that add the norms
    // in the epilogue screen groups of four centers (fewer ALU operations per value)
    const bool direct = rp.parts == 0 && (c.d & 3) == 0 &&
                        ((reinterpret_cast<uintptr_t>(c.X) | reinterpret_cast<uintptr_t>(C)) & 15u) == 0;
    p.group = (direct && tc::tc_norms_in_epilogue(fmt)) ? 4 : 2;
    ScreenBound sb{};
    sb.xnorm = c.tc_xnorm; sb.cmax_bits = c.tc_cmax; sb.st = c.st;
    sb.fix_rows = c.fix_rows; sb.fix_cnt = c.fix_cnt; sb.ub = c.tc_ub;
    tc::tc_bound(c.d, fmt, &sb.ep, &sb.en, &sb.ec);
    // a round pass whose rows already have a nearest distance D^2 lists, in the
    // screening pass itself, every center within that distance (plus the bound):
    // the rows the groups leave undecided then need no second screening
    // (Not in the first round: its rows' D^2 is the distance to the first center alone,
    // far above the spread of any cluster, so their lists would only overflow.)
    const bool plist = mode_round && p.group == 4 && c.tc_list && c.rounds_done >= 1;
    if (plist) {
        if ((e = tc::launch_row_thresholds(c.D2, c.n, c.d, c.tc_xnorm, c.tc_cmax, sb.ep, sb.en, sb.ec, c.tc_thr,
                                           c.stream)) != cudaSuccess)
            return e;
        p.thr = c.tc_thr; p.lst = c.tc_lst; p.lcnt = c.tc_lcnt;
    }
    if (rows) {
        // the compact image of the listed rows (their scales too; the thresholds the
        // gather also writes are not used by the pair epilogue)
        if (mode_round || !direct || p.group != 4 || !c.tc_cimg) return cudaErrorInvalidValue;
        if ((e = tc::launch_gather_rows(c.tc_ximg, c.tc_xscale, c.d, fmt, rows, rows_cnt, c.tc_ub, c.tc_xnorm,
                                        c.tc_cmax, sb.ep, sb.en, sb.ec, c.tc_cimg, c.tc_cscale, c.tc_thr,
                                        c.num_sms * 8, c.stream)) != cudaSuccess)
            return e;
        p.ximg = c.tc_cimg; p.xscale = c.tc_cscale; p.nrows_dev = rows_cnt;
        if ((e = tc::launch_nearest_tc(p, 0, tc::EPI_PAIR, c.num_sms, c.stream)) != cudaSuccess) return e;
        refine_direct_kernel<MODE_ASSIGN, 4><<<(int)((c.n + 255) / 256), 256, 0, c.stream>>>(
            c.X, c.n, c.d, C, k, c.cand1, c.tc_v2, sb, nullptr, nullptr, labels, prev, changed, dmin,
            &c.st->argmin_fp64, &c.st->argmin_wide, rows, rows_cnt, c.ll_ub, c.ll_lb);
        count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else {
    cudaEvent_t ev = nullptr;
    if ((e = timing_begin(c, &ev)) != cudaSuccess) return e;
    if ((e = tc::launch_nearest_tc(p, mode_round, plist ? tc::EPI_PAIRLIST : tc::EPI_PAIR, c.num_sms, c.stream)) !=
        cudaSuccess)
        return e;
    if ((e = timing_end(c, ev, timing_cls)) != cudaSuccess) return e;
    if (rp.parts > 0) {
        const int rw = rp.warps;
        const size_t rsm = resident_smem_bytes(rp.hold, c.d, rw);
        const int64_t nb = (c.n + 31) / 32;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(c.num_sms, (nb + rw - 1) / rw));
        for (int part = 0; part < rp.parts; ++part) {
            const int lo = part * rp.rows;
            if (mode_round)
                refine_resident_kernel<MODE_ROUND><<<grid, 32 * rw, rsm, c.stream>>>(
                    c.X, c.n, c.d, C, cap_rows, lo, rp.rows, rp.hold, c.cand1, c.tc_v2, sb, c.D2, c.idx, nullptr,
                    nullptr, nullptr, nullptr, &c.st->argmin_fp64, &c.st->argmin_wide);
            else
                refine_resident_kernel<MODE_ASSIGN><<<grid, 32 * rw, rsm, c.stream>>>(
                    c.X, c.n, c.d, C, cap_rows, lo, rp.rows, rp.hold, c.cand1, c.tc_v2, sb, nullptr, nullptr, labels,
                    prev, changed, dmin, &c.st->argmin_fp64, &c.st->argmin_wide);
            count_launches(1);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    } else if (direct) {
        const int grid = (int)((c.n + 255) / 256);
#define KMP_DIRECT(G)                                                                                           \
    if (mode_round)                                                                                             \
        refine_direct_kernel<MODE_ROUND, G><<<grid, 256, 0, c.stream>>>(c.X, c.n, c.d, C, 0, c.cand1, c.tc_v2, sb, \
                                                                        c.D2, c.idx, nullptr, nullptr, nullptr,  \
                                                                        nullptr, &c.st->argmin_fp64,             \
                                                                        &c.st->argmin_wide, nullptr, nullptr,    \
                                                                        nullptr, nullptr);                       \
    else                                                                                                        \
        refine_direct_kernel<MODE_ASSIGN, G><<<grid, 256, 0, c.stream>>>(c.X, c.n, c.d, C, k, c.cand1, c.tc_v2,  \
                                                                         sb, nullptr, nullptr, labels, prev,     \
                                                                         changed, dmin, &c.st->argmin_fp64,      \
                                                                         &c.st->argmin_wide, c.refine_order,     \
                                                                         nullptr, c.ll_ub, c.ll_lb);
        if (p.group == 4) { KMP_DIRECT(4) } else { KMP_DIRECT(2) }
#undef KMP_DIRECT
        count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else {
        const int rthreads = 32 * refine_warps(c.d);
        const int grid = (int)((c.n + rthreads - 1) / rthreads);
        const size_t rsm = refine_smem_bytes(c.d);
        if (mode_round)
            refine_kernel<MODE_ROUND><<<grid, rthreads, rsm, c.stream>>>(c.X, c.n, c.d, C, 0, c.cand1, c.tc_v2, sb,
                                                                         c.D2, c.idx, nullptr, nullptr, nullptr,
                                                                         nullptr, &c.st->argmin_fp64,
                                                                         &c.st->argmin_wide);
        else
            refine_kernel<MODE_ASSIGN><<<grid, rthreads, rsm, c.stream>>>(c.X, c.n, c.d, C, k, c.cand1, c.tc_v2, sb,
                                                                          nullptr, nullptr, labels, prev, changed,
                                                                          dmin, &c.st->argmin_fp64,
                                                                          &c.st->argmin_wide);
        count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    }
    if (!c.tc_list) {
        if ((e = count_fixups(c, nullptr, rows_cnt)) != cudaSuccess) return e;
        return launch_fixup(c, mode_round, C, k, labels, prev, changed, dmin, c.fix_rows, c.fix_cnt);
    }
    const int lgrid = c.num_sms * 8;
    // rows the pair screening left undecided (rows_in, cnt_in): a second screening of
    // just those rows that lists every center within twice the screening bound of
    // the row's deciding distance, the exact FP32 form of the listed centers, and the
    // exact scan only for rows whose lists overflowed or stayed uncertain (rows_out)
    auto list_pass = [&](int32_t *rows_in, int *cnt_in, int32_t *rows_out, int *cnt_out) -> cudaError_t {
        cudaError_t e2;
        if ((e2 = cudaMemsetAsync(cnt_out, 0, sizeof(int), c.stream)) != cudaSuccess) return e2;
        if ((e2 = tc::launch_gather_rows(c.tc_ximg, c.tc_xscale, c.d, fmt, rows_in, cnt_in, c.tc_ub, c.tc_xnorm,
                                         c.tc_cmax, sb.ep, sb.en, sb.ec, c.tc_cimg, c.tc_cscale, c.tc_thr,
                                         c.num_sms * 8, c.stream)) != cudaSuccess)
            return e2;
        tc::TcParams pl = p;
        pl.ximg = c.tc_cimg; pl.xscale = c.tc_cscale;
        pl.nrows_dev = cnt_in; pl.thr = c.tc_thr; pl.lst = c.tc_lst; pl.lcnt = c.tc_lcnt;
        if ((e2 = tc::launch_nearest_tc(pl, mode_round, tc::EPI_LIST, c.num_sms, c.stream)) != cudaSuccess) return e2;
        if (mode_round)
            refine_list_kernel<MODE_ROUND, false><<<lgrid, 256, 0, c.stream>>>(
                c.X, c.d, C, 0, rows_in, cnt_in, c.tc_lst, c.tc_lcnt, c.tc_thr, sb, rows_out, cnt_out, c.D2, c.idx,
                nullptr, nullptr, nullptr, nullptr, &c.st->argmin_fp64, &c.st->argmin_wide);
        else
            refine_list_kernel<MODE_ASSIGN, false><<<lgrid, 256, 0, c.stream>>>(
                c.X, c.d, C, k, rows_in, cnt_in, c.tc_lst, c.tc_lcnt, c.tc_thr, sb, rows_out, cnt_out, nullptr,
                nullptr, labels, prev, changed, dmin, &c.st->argmin_fp64, &c.st->argmin_wide);
        count_launches(1);
        return cudaGetLastError();
    };
    if (!plist) {
        if ((e = list_pass(c.fix_rows, c.fix_cnt, c.fix_rows2, c.fix_cnt2)) != cudaSuccess) return e;
        if ((e = count_fixups(c, c.fix_cnt2, rows_cnt)) != cudaSuccess) return e;
        return launch_fixup(c, mode_round, C, k, labels, prev, changed, dmin, c.fix_rows2, c.fix_cnt2);
    }
    // the lists the screening pass kept: the exact FP32 form of the listed centers;
    // rows whose lists overflowed or stayed uncertain take the list pass, and the
    // rows that one leaves, the exact scan
    if ((e = cudaMemsetAsync(c.fix_cnt2, 0, sizeof(int), c.stream)) != cudaSuccess) return e;
    refine_list_kernel<MODE_ROUND, true><<<lgrid, 256, 0, c.stream>>>(
        c.X, c.d, C, 0, c.fix_rows, c.fix_cnt, c.tc_lst, c.tc_lcnt, c.tc_thr, sb, c.fix_rows2, c.fix_cnt2, c.D2, c.idx,
        nullptr, nullptr, nullptr, nullptr, &c.st->argmin_fp64, &c.st->argmin_wide);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    count_stage_kernel<<<1, 1, 0, c.stream>>>(c.fix_cnt, nullptr, c.n, c.st);
    count_launches(1);
    if ((e = list_pass(c.fix_rows2, c.fix_cnt2, c.fix_rows, c.fix_cnt)) != cudaSuccess) return e;
    count_stage_kernel<<<1, 1, 0, c.stream>>>(nullptr, c.fix_cnt, c.n, c.st);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_fixup(c, mode_round, C, k, labels, prev, changed, dmin, c.fix_rows, c.fix_cnt);
}

// ---------------------------------------------------------------- Lloyd's bounds
// Between Lloyd iterations every center c moves by delta_c = ||c_new - c_old||.
// A row labelled a with u >= d(x, c_a) and l <= d(x, c) for every other c keeps
// u + delta_a and l - max_{c != a} delta_c as bounds for the moved centers (the
// triangle inequality); if the first is below the second, a is still strictly the
// nearest center, by more than the FP32 tie window (both bounds carry it), so the
// exact FP32 argmin takes a again and only d^2(x, c_a) needs computing.

// delta_c in FP64 from the FP32 centers, rounded up to FP32 (one warp per center)
__global__ void lloyd_drift_kernel(const float *__restrict__ Cn, const float *__restrict__ Co, int k, int d,
                                   float *__restrict__ drift) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= k) return;
    double s = 0.0;
    for (int q = lane; q < d; q += 32) {
        const double t = (double)Cn[(size_t)c * d + q] - (double)Co[(size_t)c * d + q];
        s = __fma_rn(t, t, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) drift[c] = __double2float_ru(sqrt(s));
}

// for every center, the largest drift among the other centers (one block)
__global__ void __launch_bounds__(1024) lloyd_drift_other_kernel(const float *__restrict__ drift, int k,
                                                                 float *__restrict__ other) {
    __shared__ float s1[32], s2[32];
    __shared__ int si[32];
    float m1 = 0.f, m2 = 0.f;
    int i1 = -1;
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        const float v = drift[c];
        if (v > m1) { m2 = m1; m1 = v; i1 = c; }
        else if (v > m2) m2 = v;
    }
    // merge the top two of the warp, then of the block
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float a1 = __shfl_xor_sync(0xffffffffu, m1, o), a2 = __shfl_xor_sync(0xffffffffu, m2, o);
        const int ai = __shfl_xor_sync(0xffffffffu, i1, o);
        if (a1 > m1 || (a1 == m1 && ai < i1)) { m2 = fmaxf(m1, a2); m1 = a1; i1 = ai; }
        else m2 = fmaxf(m2, a1);
    }
    if (lane == 0) { s1[wid] = m1; s2[wid] = m2; si[wid] = i1; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        m1 = lane < nw ? s1[lane] : 0.f;
        m2 = lane < nw ? s2[lane] : 0.f;
        i1 = lane < nw ? si[lane] : -1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float a1 = __shfl_xor_sync(0xffffffffu, m1, o), a2 = __shfl_xor_sync(0xffffffffu, m2, o);
            const int ai = __shfl_xor_sync(0xffffffffu, i1, o);
            if (a1 > m1 || (a1 == m1 && ai < i1)) { m2 = fmaxf(m1, a2); m1 = a1; i1 = ai; }
            else m2 = fmaxf(m2, a1);
        }
        if (lane == 0) { s1[0] = m1; s2[0] = m2; si[0] = i1; }
    }
    __syncthreads();
    m1 = s1[0]; m2 = s2[0]; i1 = si[0];
    for (int c = threadIdx.x; c < k; c += blockDim.x) other[c] = c == i1 ? m2 : m1;
}

// The bounds test for every row (in the order given: rows sorted by their previous
// label, so neighbouring threads read the same center row).  A row it settles gets
// its label, the exact FP32 d^2 to the moved center (bit-identical to the refine's
// chains) and fresh bounds; the others are listed for the compact pass (with l = 0
// until that pass certifies them again).
__global__ void __launch_bounds__(256) lloyd_bounds_kernel(const float *__restrict__ X, int64_t n, int d,
                                                           const float *__restrict__ C,
                                                           const int32_t *__restrict__ prev,
                                                           const int32_t *__restrict__ order, int32_t *labels,
                                                           float *dmin, float *ubd, float *lbd,
                                                           const float *__restrict__ drift,
                                                           const float *__restrict__ other, int32_t *rows, int *cnt,
                                                           unsigned long long *settled) {
    const int64_t T = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = T < n;
    const int64_t R = order && valid ? (int64_t)order[T] : T;
    const int lane = threadIdx.x & 31;
    bool keep = false;
    if (valid) {
        const int a = prev[R];
        const float u = ubd[R] + drift[a];
        const float l = lbd[R] - other[a];
        keep = l > 0.f && u < l;
        if (keep) {
            const float4 *x4 = reinterpret_cast<const float4 *>(X + R * d);
            const float4 *c4 = reinterpret_cast<const float4 *>(C + (int64_t)a * d);
            float v = 0.f;
#pragma unroll 4
            for (int p = 0; p < (d >> 2); ++p) {
                const float4 x = __ldg(x4 + p), c = __ldg(c4 + p);
                float t;
                t = __fsub_rn(x.x, c.x); v = __fmaf_rn(t, t, v);
                t = __fsub_rn(x.y, c.y); v = __fmaf_rn(t, t, v);
                t = __fsub_rn(x.z, c.z); v = __fmaf_rn(t, t, v);
                t = __fsub_rn(x.w, c.w); v = __fmaf_rn(t, t, v);
            }
            labels[R] = a;
            dmin[R] = v;
            ubd[R] = bound_upper(v, fp32_tie_window(d));
            lbd[R] = l;
        } else {
            lbd[R] = 0.f;
        }
    }
    const unsigned m = __ballot_sync(0xffffffffu, valid && !keep);
    if (m) {
        int base = 0;
        if (lane == 0) base = atomicAdd(cnt, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (valid && !keep) rows[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)R;
    }
    const unsigned kp = __ballot_sync(0xffffffffu, keep);
    if (lane == 0 && kp) atomicAdd(settled, (unsigned long long)__popc(kp));
}

bool lloyd_bounds_usable(const Ctx &c, const float *C) {
    if (c.precision == KMPAR_FP32 || !c.ll_lb || !c.tc_cimg) return false;
    const ResidentPlan rp = resident_plan(c.k, c.d);
    return rp.parts == 0 && (c.d & 3) == 0 && tc::tc_norms_in_epilogue(c.tc_fmt) &&
           ((reinterpret_cast<uintptr_t>(c.X) | reinterpret_cast<uintptr_t>(C)) & 15u) == 0;
}

// one Lloyd assignment after a centroid update, using the bounds: the rows they
// settle, then a compact tensor pass over the rest
cudaError_t launch_lloyd_bounded_pass(Ctx &c, const float *C, int32_t *labels, const int32_t *prev, int *changed,
                                      float *dmin) {
    cudaError_t e;
    const int k = c.k;
    lloyd_drift_kernel<<<(k + 7) / 8, 256, 0, c.stream>>>(C, c.ll_cold, k, c.d, c.ll_drift);
    lloyd_drift_other_kernel<<<1, 1024, 0, c.stream>>>(c.ll_drift, k, c.ll_other);
    count_launches(2);
    if ((e = cudaMemsetAsync(c.ll_cnt, 0, sizeof(int), c.stream)) != cudaSuccess) return e;
    // rows in storage order: X streams from HBM, the settled rows' center rows (k x d,
    // a few MB) come from L2
    lloyd_bounds_kernel<<<(int)((c.n + 255) / 256), 256, 0, c.stream>>>(
        c.X, c.n, c.d, C, prev, nullptr, labels, dmin, c.ll_ub, c.ll_lb, c.ll_drift, c.ll_other, c.ll_rows, c.ll_cnt,
        &c.st->lloyd_settled);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_tc_pass(c, 0, C, k, labels, prev, changed, dmin, -1, c.ll_rows, c.ll_cnt);
}

}  // namespace kmp
