// nearest_tc.cuh -- parameters and launchers of the tcgen05 screening passes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kmp {
struct DevState;
namespace tc {

// Operand formats of the screening GEMM.  In the BF16 and BF16X3 formats
// ||c'||^2 rides in two extra K columns; in BF16N and FP8 the K columns hold the
// coordinates only and the epilogue adds ||c'||^2 with one FMA per value.
enum Fmt {
    FMT_BF16 = 0,    // A [x', 1, 1], B [-2c', cn_hi, cn_lo], BF16
    FMT_BF16X3 = 1,  // split hi/lo BF16, three products
    FMT_BF16N = 2,   // A [x'], B [c'], BF16, norms in the epilogue
    FMT_FP8 = 3      // A e4m3(x' / s_x) per-row power-of-two scale, B e4m3(c' / s_t) per center tile
};

// what the epilogue keeps per row
enum Epi {
    EPI_PAIR = 0,     // the best pair of adjacent centers and the best screened value outside it
    EPI_LIST = 1,     // every center whose screened value is at most the row's threshold
    EPI_PAIRLIST = 2  // both (groups of four): the pair result and the list, for every row
};

constexpr int kListSlots = 8;   // list entries per row and column group (4 groups per row)

struct TcParams {
    const float *X;          // n x d FP32 points
    int64_t n;               // rows (EPI_PAIR); EPI_LIST reads the count from nrows_dev
    int d;
    int fmt;
    const uint8_t *ximg;     // swizzled image of X (or of the listed rows), one block per 128-row tile
    const float *xnorm;      // ||x'||^2 per point (FP32, x' = x - anchor)
    const float *xscale;     // FP8: per-row scale s_x of the A image
    const float *Cf;         // FP32 center rows (ROUND: candidate matrix; ASSIGN: k centers)
    int cnt;                 // ASSIGN: number of centers
    const DevState *st;      // ROUND: batch range
    const uint8_t *bimg;     // swizzled center tiles
    const float *ncol;       // BF16N / FP8: ||c'||^2 per pass-local center (pad rows: 1e30)
    const float *tscale;     // BF16N / FP8: per center tile scale (1 for BF16N)
    const unsigned int *cmax_bits;
    int32_t *cand1;          // EPI_PAIR: per row, first center of the best screened group (-1: none)
    float *v2;               // EPI_PAIR: per row, smallest screened value outside that group (key-truncated)
    const int *nrows_dev;    // EPI_LIST: number of listed rows (EPI_PAIR: of a compact image's rows, or null: n)
    const float *thr;        // EPI_LIST: per listed row (EPI_PAIRLIST: per row), the screened-value threshold
    int32_t *lst;            // EPI_LIST / EPI_PAIRLIST: per row, 4 x kListSlots pass-local center numbers
    int32_t *lcnt;           // per row and group, entries found (> kListSlots: overflow)
    int32_t *fix_rows;       // rows left to the exact CUDA-core pass
    int *fix_cnt;
    unsigned long long *fp64_cnt;
    int *err;                // first timeout code, 0 if none
    int group;               // EPI_PAIR: centers per screened group, 2 or 4 (BF16N and FP8 only)
    int ksteps;              // MMA instructions per tile (32 bytes of K each)
    uint32_t vmask;          // value bits of a key (set by launch_nearest_tc)
};

// screening format of a precision mode at dimension d (-1: not built)
int tc_format(int precision, int d);
bool tc_supported(int d, int fmt);
int tc_katoms(int d, int fmt);
int tc_ksteps(int d, int fmt);
int tc_block_n(int d, int fmt);
bool tc_norms_in_epilogue(int fmt);
size_t tc_image_bytes(int d, int fmt, int cap_rows);
size_t tc_points_image_bytes(int d, int fmt, int64_t n);
int tc_center_tiles(int d, int fmt, int cap_rows);
// column means of X (d floats), the anchor the screening operands are moved by;
// scratch holds tc_anchor_scratch_doubles(d) doubles
size_t tc_anchor_scratch_doubles(int d);
cudaError_t launch_anchor(const float *X, int64_t n, int d, double *scratch, float *anchor, cudaStream_t s);
cudaError_t launch_prep_points(const float *X, int64_t n, int d, int fmt, const float *anchor, uint8_t *img,
                               float *xnorm, float *xscale, cudaStream_t s);
cudaError_t launch_prep_centers(const float *C, int d, int fmt, const DevState *st, int cnt_static, int round_mode,
                                int cap_rows, const float *anchor, uint8_t *img, float *ncol, float *tscale,
                                unsigned int *cmax_bits, cudaStream_t s);
cudaError_t launch_nearest_tc(TcParams p, int mode_round, int epi, int num_sms, cudaStream_t s);
// Rows listed in rows[0 .. *cnt) gathered into a compact image (row i of the compact
// image = image row rows[i]), with their scales and list thresholds
// thr[i] = ub[rows[i]] - ||x'||^2 + T, T covering twice the screening bound and the
// FP32 tie window (see the list pass).
cudaError_t launch_gather_rows(const uint8_t *img, const float *xscale, int d, int fmt, const int32_t *rows,
                               const int *cnt, const float *ub, const float *xnorm, const unsigned int *cmax_bits,
                               float ep, float en, float ec, uint8_t *cimg, float *cscale, float *thr, int grid,
                               cudaStream_t s);
// screening error bound E(x, c) = ep ||x'|| ||c'|| + en (||x'||^2 + ||c'||^2) + ec ||x'|| max ||c'||
void tc_bound(int d, int fmt, float *ep, float *en, float *ec);
// per row R < n, the list threshold of a row whose nearest distance is at most ub[R]
// (the same threshold as launch_gather_rows writes for a listed row)
cudaError_t launch_row_thresholds(const float *ub, int64_t n, int d, const float *xnorm,
                                  const unsigned int *cmax_bits, float ep, float en, float ec, float *thr,
                                  cudaStream_t s);

}  // namespace tc
}  // namespace kmp
