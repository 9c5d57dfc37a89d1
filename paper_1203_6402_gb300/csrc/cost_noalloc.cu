// cost_noalloc.cu -- kmpar_cost_noalloc: phi_X(C) with no device allocation.
//
// The per-block FP64 partial sums, the final sum and a statistics counter live in
// one file-scope device array (kNoAllocScratchDoubles doubles, 512 KB + 24 B),
// which every GPU that loads the library holds until the process exits.  Host
// code cannot use the array's name as a device address, so every call looks the
// address up with cudaGetSymbolAddress on the current device (the lookup
// allocates nothing); nothing is cached, so a call after cudaDeviceReset, or
// from another context, still gets the array of the context it runs in.  All
// calls share the array: calls whose kernels overlap on the GPU race on it.
#include "kmpar_internal.cuh"

namespace kmp {
void set_thread_error(const std::string &m);   // read back by kmpar_last_error(NULL)
}

constexpr int kNoAllocMaxBlocks = 65536;                      // per-block partials
constexpr int kNoAllocScratchDoubles = kNoAllocMaxBlocks + 3; // + sum + counter (+ pad)

static __device__ __align__(256) double g_cost_scratch[kNoAllocScratchDoubles];

namespace {

kmpar_status noalloc_fail(kmpar_status s, const std::string &m) {
    kmp::set_thread_error(m);
    return s;
}

// device address of g_cost_scratch in the current context, looked up on every
// call (no cache that a device reset or a context switch could leave stale)
cudaError_t scratch_address(double **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_cost_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<double *>(p);
    return cudaSuccess;
}

}  // namespace

extern "C" {

kmpar_status kmpar_cost_noalloc(const float *X, int64_t n, int32_t d, const float *C, int32_t k, double *phi,
                                void *stream) {
    if (!X || !C || !phi) return noalloc_fail(KMPAR_ERR_ARG, "NULL pointer");
    if (n < 1 || d < 1 || d > 4096 || k < 1) return noalloc_fail(KMPAR_ERR_ARG, "size out of range");
    const int np = kmp::assign_num_partials(n, d);
    if (n > (int64_t)kNoAllocMaxBlocks * 128 || np > kNoAllocMaxBlocks)
        return noalloc_fail(KMPAR_ERR_ARG, "n exceeds the 8,388,608-point limit of kmpar_cost_noalloc");
    cudaStream_t s = (cudaStream_t)stream;
    double *buf = nullptr;
    cudaError_t e = scratch_address(&buf);
    if (e != cudaSuccess) return noalloc_fail(KMPAR_ERR_CUDA, std::string("scratch address: ") + cudaGetErrorString(e));
    double *sum = buf + kNoAllocMaxBlocks;
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(buf + kNoAllocMaxBlocks + 1);
    // the counter accumulates across a call, so it starts from zero; every partial
    // and the sum are overwritten by each call
    e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = kmp::launch_assign(X, n, d, C, k, nullptr, nullptr, nullptr, buf, np, cnt, s);
    if (e == cudaSuccess) e = kmp::launch_sum_f64(buf, np, sum, nullptr, s);
    double h = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sum, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_fail(KMPAR_ERR_CUDA, std::string("cost kernels: ") + cudaGetErrorString(e));
    *phi = h;
    return KMPAR_OK;
}

}  // extern "C"
