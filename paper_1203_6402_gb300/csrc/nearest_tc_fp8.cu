// nearest_tc_fp8.cu -- the screening pass (nearest_tc_kernel.cuh) instantiated for
// the FMT_FP8 operand format; one translation unit per format keeps the build parallel.
#include "nearest_tc_kernel.cuh"

namespace kmp {
namespace tc {

cudaError_t dispatch_fp8(const TcParams &p, int mode_round, int epi, int KA, int grid, cudaStream_t s) {
    if (epi == EPI_LIST) return dispatch_fmt<FMT_FP8, EPI_LIST>(p, mode_round, KA, grid, s);
    if (epi == EPI_PAIRLIST) return dispatch_fmt<FMT_FP8, EPI_PAIRLIST, 4>(p, mode_round, KA, grid, s);
    if (p.group == 4) return dispatch_fmt<FMT_FP8, EPI_PAIR, 4>(p, mode_round, KA, grid, s);
    return dispatch_fmt<FMT_FP8, EPI_PAIR>(p, mode_round, KA, grid, s);
}

}  // namespace tc
}  // namespace kmp
