// nearest_tc.cuh -- parameters and launchers of the tcgen05 screening pass.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kmp {
struct DevState;
namespace tc {

struct TcParams {
    const float *X;          // n x d FP32 points
    int64_t n;
    int d;
    int split;               // 0: BF16, 1: split BF16 (hi/lo, three products)
    const uint8_t *ximg;     // swizzled BF16 image of X, one block per 128-row tile
    const float *xnorm;      // ||x'||^2 per point (FP32, x' = x - anchor)
    const float *Cf;         // FP32 center rows (ROUND: candidate matrix; ASSIGN: k centers)
    int cnt;                 // ASSIGN: number of centers
    const DevState *st;      // ROUND: batch range
    const uint8_t *bimg;     // swizzled BF16 center tiles
    const unsigned int *cmax_bits;
    int32_t *cand1;          // per row: first center of the best screened pair (-1: none)
    float *v2;               // per row: smallest screened value outside that pair (key-truncated)
    int32_t *fix_rows;       // rows left to the exact CUDA-core pass
    int *fix_cnt;
    unsigned long long *fp64_cnt;
    int *err;                // first timeout code, 0 if none
    float ep, en;            // screening error bound coefficients
    int ksteps;              // K / 16
    uint32_t vmask;          // value bits of a key (set by launch_nearest_tc)
};

bool tc_supported(int d, int split);
int tc_katoms(int d, int split);
int tc_ksteps(int d, int split);
int tc_block_n(int d, int split);
size_t tc_image_bytes(int d, int split, int cap_rows);
size_t tc_points_image_bytes(int d, int split, int64_t n);
// column means of X (d floats), the anchor the screening operands are moved by;
// scratch holds tc_anchor_scratch_doubles(d) doubles
size_t tc_anchor_scratch_doubles(int d);
cudaError_t launch_anchor(const float *X, int64_t n, int d, double *scratch, float *anchor, cudaStream_t s);
cudaError_t launch_prep_points(const float *X, int64_t n, int d, int split, const float *anchor, uint8_t *img,
                               float *xnorm, cudaStream_t s);
cudaError_t launch_prep_centers(const float *C, int d, int split, const DevState *st, int cnt_static, int round_mode,
                                int cap_rows, const float *anchor, uint8_t *img, unsigned int *cmax_bits,
                                cudaStream_t s);
cudaError_t launch_nearest_tc(TcParams p, int mode_round, int num_sms, cudaStream_t s);
// screening error bound E(x, c) = ep ||x'|| ||c'|| + en (||x'||^2 + ||c'||^2)
void tc_bound(int d, int split, float *ep, float *en);

}  // namespace tc
}  // namespace kmp
