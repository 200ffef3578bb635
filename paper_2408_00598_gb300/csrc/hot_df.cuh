// Double-float arithmetic for the CUDA kernels of the HOT library.
//
// An unevaluated pair (hi, lo) of FP32 values whose sum carries about twice
// the FP32 precision (about 48 significant bits): the double-length arithmetic
// of Dekker (1971).  Each add is Knuth's exact two-sum (TAOCP vol. 2, 4.2.2)
// followed by renormalisation (fast two-sum); a product takes the exact
// rounding error of hi * hi from a fused multiply-add in place of Dekker's
// splitting.  FP64 arithmetic runs at a small fraction of the FP32
// rate on GB300, so sums and comparisons that must be accurate to FP64 level
// use these pairs on the FP32 pipe.
#pragma once

#include <cuda_runtime.h>

namespace hot {

struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_add(DF a, float b) {
    const float s = a.hi + b;
    const float bb = s - a.hi;
    const float e = ((a.hi - (s - bb)) + (b - bb)) + a.lo;
    const float h = s + e;
    return DF{h, e - (h - s)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF r = df_add(a, b.hi);
    return df_add(r, b.lo);
}
__device__ __forceinline__ double df_val(DF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ DF df_from(double x) {
    const float h = (float)x;
    return DF{h, (float)(x - (double)h)};
}
__device__ __forceinline__ DF df_ld(float2 v) { return DF{v.x, v.y}; }
__device__ __forceinline__ float2 df_st(DF a) { return make_float2(a.hi, a.lo); }
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ float df_f(DF a) { return a.hi + a.lo; }
// products: the error of hi*hi is exact by fma; the cross terms are FP32
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float h = p + e;
    return DF{h, e - (h - p)};
}
__device__ __forceinline__ DF df_mul(DF a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    const float h = p + e;
    return DF{h, e - (h - p)};
}
__device__ __forceinline__ DF df_shfl_down(DF a, int o) {
    return DF{__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}
// warp sum in a fixed tree; the result is valid in lane 0
__device__ __forceinline__ DF warp_sum_df(DF a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = df_add(a, df_shfl_down(a, o));
    return a;
}

}  // namespace hot
