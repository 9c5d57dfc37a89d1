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
// One CTA of 1024 threads; thread t owns the contiguous candidate range
// [t q, (t+1) q).  Per draw: FP64 masses, a fixed-order block scan, the target
// u * total, the first candidate whose running prefix exceeds it, and the D^2
// update of every candidate against the drawn one (exact FP32 difference form).
constexpr int kRcThreads = 1024;

__device__ __forceinline__ double block_incl_scan_f64(double v, double *buf) {
    const int t = threadIdx.x;
    buf[t] = v;
    __syncthreads();
    for (int off = 1; off < kRcThreads; off <<= 1) {
        const double a = t >= off ? buf[t - off] : 0.0;
        __syncthreads();
        if (t >= off) buf[t] = buf[t] + a;
        __syncthreads();
    }
    return buf[t];
}

__global__ void __launch_bounds__(kRcThreads) recluster_kernel(const float *__restrict__ C,
                                                             const long long *__restrict__ w, DevState *st,
                                                             int d, int k, uint64_t seed, float *rD2,
                                                             int32_t *chosen, float *centers) {
    __shared__ double buf[kRcThreads];
    __shared__ int s_min[32], s_max[32];
    __shared__ int s_pick;
    extern __shared__ float cnew[];
    const int m = st->m;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int q = (m + kRcThreads - 1) / kRcThreads;
    const int lo = min(m, t * q), hi = min(m, lo + q);

    for (int step = 0; step < k; ++step) {
        double local = 0.0;
        for (int j = lo; j < hi; ++j)
            local += step == 0 ? (double)w[j] : __dmul_rn((double)w[j], (double)rD2[j]);
        const double incl = block_incl_scan_f64(local, buf);
        const double excl = t > 0 ? buf[t - 1] : 0.0;
        const double total = buf[kRcThreads - 1];
        __syncthreads();
        if (!(total > 0.0)) {
            // positive mass exhausted: remaining draws repeat the first center
            for (int s = step + t; s < k; s += kRcThreads) chosen[s] = step > 0 ? chosen[0] : 0;
            if (t == 0) st->warn = 1;
            __syncthreads();
            for (int s = step; s < k; ++s) {
                const int src = step > 0 ? chosen[0] : 0;
                for (int qq = t; qq < d; qq += kRcThreads) centers[(int64_t)s * d + qq] = C[(int64_t)src * d + qq];
            }
            return;
        }
        (void)incl;
        const double u = uniform53((uint64_t)step, 0, TAG_RECLUSTER, seed);
        const double target = __dmul_rn(u, total);
        int mine = INT_MAX, lastpos = -1;
        bool nt = false;
        double run = excl;
        for (int j = lo; j < hi; ++j) {
            const double e = step == 0 ? (double)w[j] : __dmul_rn((double)w[j], (double)rD2[j]);
            const double before = run;
            run = run + e;
            if (e > 0.0) lastpos = j;
            if (mine == INT_MAX && run > target) {
                mine = j;
                nt = fabs(target - before) <= 1e-6 * total || fabs(run - target) <= 1e-6 * total;
            }
        }
        // block min of the first crossing, block max of the last positive mass
        int a = mine, b = lastpos;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = min(a, __shfl_down_sync(0xffffffffu, a, o));
            b = max(b, __shfl_down_sync(0xffffffffu, b, o));
        }
        if (lane == 0) { s_min[wid] = a; s_max[wid] = b; }
        __syncthreads();
        if (t == 0) {
            int pa = INT_MAX, pb = -1;
            for (int i = 0; i < kRcThreads / 32; ++i) { pa = min(pa, s_min[i]); pb = max(pb, s_max[i]); }
            if (pa == INT_MAX) { pa = pb; atomicAdd(&st->recluster_near, 1ull); }
            s_pick = pa;
            chosen[step] = pa;
        }
        __syncthreads();
        if (nt && mine == s_pick) atomicAdd(&st->recluster_near, 1ull);
        const int pick = s_pick;
        for (int qq = t; qq < d; qq += kRcThreads) {
            const float v = C[(int64_t)pick * d + qq];
            cnew[qq] = v;
            centers[(int64_t)step * d + qq] = v;
        }
        __syncthreads();
        for (int j = lo; j < hi; ++j) {
            const float v = dist2_fp32(C + (int64_t)j * d, cnew, d);
            rD2[j] = step == 0 ? v : fminf(rD2[j], v);
        }
        __syncthreads();
    }
}

cudaError_t launch_recluster(Ctx &c, float *centers) {
    const size_t smem = sizeof(float) * (size_t)c.d;
    recluster_kernel<<<1, kRcThreads, smem, c.stream>>>(c.C, c.w, c.st, c.d, c.k, c.seed, c.rD2, c.chosen,
                                                       centers);
    count_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Lloyd: centroids
// per sort block b (kSortBlock points): hist[b][j] = #points with label j
__global__ void label_hist_kernel(const int32_t *__restrict__ labels, int64_t n, int k, int32_t *hist) {
    extern __shared__ int32_t h[];
    for (int j = threadIdx.x; j < k; j += blockDim.x) h[j] = 0;
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * kSortBlock;
    const int64_t b1 = min(n, b0 + kSortBlock);
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) atomicAdd(&h[labels[i]], 1);
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) hist[(int64_t)blockIdx.x * k + j] = h[j];
}

// column scan: hist[b][j] <- sum_{b' < b} hist[b'][j]; tot[j] = column total
__global__ void column_scan_kernel(int32_t *hist, int nsb, int k, int32_t *tot) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    int run = 0;
    for (int b = 0; b < nsb; ++b) {
        const int v = hist[(int64_t)b * k + j];
        hist[(int64_t)b * k + j] = run;
        run += v;
    }
    tot[j] = run;
}

// base[j] = sum_{j' < j} tot[j'], base[k] = n (one CTA, contiguous chunks)
__global__ void __launch_bounds__(1024) base_scan_kernel(int32_t *tot_base, int k) {
    __shared__ int buf[1024];
    const int t = threadIdx.x;
    const int q = (k + 1023) / 1024;
    const int lo = min(k, t * q), hi = min(k, lo + q);
    int local = 0;
    for (int j = lo; j < hi; ++j) local += tot_base[j];
    buf[t] = local;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int a = t >= off ? buf[t - off] : 0;
        __syncthreads();
        buf[t] += a;
        __syncthreads();
    }
    int run = t > 0 ? buf[t - 1] : 0;
    const int total = buf[1023];
    __syncthreads();
    for (int j = lo; j < hi; ++j) {
        const int v = tot_base[j];
        tot_base[j] = run;
        run += v;
    }
    if (t == 0) tot_base[k] = total;
}

// one warp per sort block: stable scatter of point numbers into label order
__global__ void __launch_bounds__(32) scatter_kernel(const int32_t *__restrict__ labels, int64_t n, int k,
                                                     const int32_t *__restrict__ hist,
                                                     const int32_t *__restrict__ base, int32_t *perm) {
    extern __shared__ int32_t cur[];
    const int lane = threadIdx.x;
    for (int j = lane; j < k; j += 32) cur[j] = base[j] + hist[(int64_t)blockIdx.x * k + j];
    __syncwarp();
    const int64_t b0 = (int64_t)blockIdx.x * kSortBlock;
    const int64_t b1 = min(n, b0 + kSortBlock);
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

// one CTA (8 warps) per cluster: FP64 sum of member rows in a fixed order, then
// centroid = sum / count rounded to FP32; an empty cluster keeps its center.
__global__ void __launch_bounds__(256) centroid_kernel(const float *__restrict__ X, int d,
                                                       const int32_t *__restrict__ perm,
                                                       const int32_t *__restrict__ base, float *centers) {
    __shared__ double part[8][32];
    const int j = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int b0 = base[j], cnt = base[j + 1] - b0;
    if (cnt == 0) return;
    for (int dc = 0; dc < d; dc += 32) {
        const int q = dc + lane;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        if (q < d) {
            int p = wid;
            for (; p + 24 < cnt; p += 32) {
                a0 += (double)X[(int64_t)perm[b0 + p] * d + q];
                a1 += (double)X[(int64_t)perm[b0 + p + 8] * d + q];
                a2 += (double)X[(int64_t)perm[b0 + p + 16] * d + q];
                a3 += (double)X[(int64_t)perm[b0 + p + 24] * d + q];
            }
            for (; p < cnt; p += 8) a0 += (double)X[(int64_t)perm[b0 + p] * d + q];
        }
        part[wid][lane] = (a0 + a1) + (a2 + a3);
        __syncthreads();
        if (wid == 0 && q < d) {
            double s = 0.0;
            for (int w8 = 0; w8 < 8; ++w8) s += part[w8][lane];
            centers[(int64_t)j * d + q] = (float)__ddiv_rn(s, (double)cnt);
        }
        __syncthreads();
    }
}

cudaError_t launch_centroids(Ctx &c, const int32_t *labels, float *centers) {
    cudaError_t e;
    const int k = c.k;
    label_hist_kernel<<<c.nsb, 256, sizeof(int32_t) * k, c.stream>>>(labels, c.n, k, c.hist);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    column_scan_kernel<<<(k + 255) / 256, 256, 0, c.stream>>>(c.hist, c.nsb, k, c.base);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    base_scan_kernel<<<1, 1024, 0, c.stream>>>(c.base, k);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    scatter_kernel<<<c.nsb, 32, sizeof(int32_t) * k, c.stream>>>(labels, c.n, k, c.hist, c.base, c.perm);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    centroid_kernel<<<k, 256, 0, c.stream>>>(c.X, c.d, c.perm, c.base, centers);
    count_launches(5);
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
