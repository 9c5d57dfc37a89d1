// dfloat.cuh -- masses and prefix sums as unevaluated sums of two floats
// (hi + lo, about 48 significant bits), used by the weighted k-means++ kernels.
// A product w D^2 is exact (w split into two floats whose sum is exact, the
// product's rounding error recovered with an FMA) and each addition carries its
// rounding error (Knuth's two-sum), so a sum of N masses is within ~N 2^-48 of its
// exact value.  FP64 arithmetic runs at a small fraction of the FP32 rate on this
// part; these sums stay on the FP32 pipes.
#pragma once

#include <cuda_runtime.h>

namespace kmp {

struct Df {
    float hi, lo;
};
__device__ __forceinline__ Df df_add(Df a, Df b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bv = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bv)), __fsub_rn(b.hi, bv));
    const float t = __fadd_rn(__fadd_rn(a.lo, b.lo), err);
    const float hi = __fadd_rn(s, t);
    return {hi, __fsub_rn(t, __fsub_rn(hi, s))};
}
// the mass of a candidate: w (first draw) or w D^2, with w = wv.x + wv.y exactly
__device__ __forceinline__ Df df_mass(float2 wv, float d2, bool first) {
    if (first) return {wv.x, wv.y};
    const float p = __fmul_rn(wv.x, d2);
    const float lo = __fmaf_rn(wv.y, d2, __fmaf_rn(wv.x, d2, -p));   // (wv.x d2 - p) exactly, + wv.y d2
    const float hi = __fadd_rn(p, lo);
    return {hi, __fsub_rn(lo, __fsub_rn(hi, p))};
}
__device__ __forceinline__ Df warp_incl_scan_df(Df v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Df u = {__shfl_up_sync(0xffffffffu, v.hi, o), __shfl_up_sync(0xffffffffu, v.lo, o)};
        if (lane >= o) v = df_add(u, v);
    }
    return v;
}
__device__ __forceinline__ double df_to_double(Df a) { return (double)a.hi + (double)a.lo; }


// the two floats of an int64 weight w < 2^48: hi = w rounded, lo = the exact rest
__device__ __forceinline__ float2 weight_split(long long w) {
    const float hi = __ll2float_rn(w);
    return make_float2(hi, __ll2float_rn(w - __float2ll_rn(hi)));
}

}  // namespace kmp
