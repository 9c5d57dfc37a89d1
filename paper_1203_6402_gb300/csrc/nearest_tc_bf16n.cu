// nearest_tc_bf16n.cu -- the screening pass (nearest_tc_kernel.cuh) instantiated for
// the FMT_BF16N operand format; one translation unit per format keeps the build parallel.
#include "nearest_tc_kernel.cuh"

namespace kmp {
namespace tc {

cudaError_t dispatch_bf16n(const TcParams &p, int mode_round, int epi, int KA, int grid, cudaStream_t s) {
    if (epi == EPI_LIST) return dispatch_fmt<FMT_BF16N, EPI_LIST>(p, mode_round, KA, grid, s);
    if (epi == EPI_PAIRLIST) return dispatch_fmt<FMT_BF16N, EPI_PAIRLIST, 4>(p, mode_round, KA, grid, s);
    if (p.group == 4) return dispatch_fmt<FMT_BF16N, EPI_PAIR, 4>(p, mode_round, KA, grid, s);
    return dispatch_fmt<FMT_BF16N, EPI_PAIR>(p, mode_round, KA, grid, s);
}

}  // namespace tc
}  // namespace kmp
