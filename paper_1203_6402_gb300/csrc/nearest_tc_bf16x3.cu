// nearest_tc_bf16x3.cu -- the screening pass (nearest_tc_kernel.cuh) instantiated for
// the FMT_BF16X3 operand format; one translation unit per format keeps the build parallel.
#include "nearest_tc_kernel.cuh"

namespace kmp {
namespace tc {

cudaError_t dispatch_bf16x3(const TcParams &p, int mode_round, int epi, int KA, int grid, cudaStream_t s) {
    if (epi == EPI_LIST) return cudaErrorInvalidValue;   // the split format has no list pass
    if (epi == EPI_PAIRLIST) return cudaErrorInvalidValue;   // groups of four only
    return dispatch_fmt<FMT_BF16X3, EPI_PAIR>(p, mode_round, KA, grid, s);
}

}  // namespace tc
}  // namespace kmp
