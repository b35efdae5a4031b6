// df64.cuh -- double-float arithmetic on the FP32 pipe.
//
// GB300 executes FP64 at about 1/64 of its FP32 rate, so a streaming kernel that performs more
// than ~2 FP64 instructions (conversions included) per cell is bound by the FP64 pipe instead of
// HBM.  Quantities that need FP64-level accuracy in the mixed-precision path (velocity state,
// Poisson right-hand side and solution, Welford accumulators, dot products) are therefore held
// as unevaluated sums hi + lo of two floats (|lo| <= ulp(hi)/2, about 48 significant bits) and
// combined with the error-free transformations of Knuth (TwoSum), Dekker (FastTwoSum) and the
// FMA-based TwoProduct.
#pragma once
#include <cuda_runtime.h>

namespace envar {

struct f2 {
    float h, l;
};

__device__ __forceinline__ f2 two_sum(float a, float b)
{
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ f2 fast_two_sum(float a, float b)   // requires |a| >= |b| or a == 0
{
    float s = a + b;
    float e = b - (s - a);
    return {s, e};
}
__device__ __forceinline__ f2 two_prod(float a, float b)
{
    float p = a * b;
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ f2 df_add(f2 a, f2 b)
{
    f2 s = two_sum(a.h, b.h);
    float e = s.l + (a.l + b.l);
    return fast_two_sum(s.h, e);
}
__device__ __forceinline__ f2 df_sub(f2 a, f2 b) { return df_add(a, f2{-b.h, -b.l}); }
__device__ __forceinline__ f2 df_add_f(f2 a, float b)
{
    f2 s = two_sum(a.h, b);
    return fast_two_sum(s.h, s.l + a.l);
}
__device__ __forceinline__ f2 df_mul(f2 a, f2 b)
{
    float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ f2 df_mul_f(f2 a, float b)
{
    float p = a.h * b;
    float e = fmaf(a.h, b, -p);
    e = fmaf(a.l, b, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ f2 df_scale_half(f2 a) { return {0.5f * a.h, 0.5f * a.l}; }
__device__ __forceinline__ double df_to_d(f2 a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ double to_dbl(f2 a) { return df_to_d(a); }
__device__ __forceinline__ f2 d_to_df(double d)
{
    float h = (float)d;
    return {h, (float)(d - (double)h)};
}
// 1/n for a positive integer n, to df64 accuracy (one Newton step on the float reciprocal).
__device__ __forceinline__ f2 df_recip_int(int n)
{
    float fn = (float)n;                 // exact for n < 2^24
    float r = 1.0f / fn;
    float e = fmaf(-fn, r, 1.0f);        // exact residual 1 - n r
    return fast_two_sum(r, r * e);
}

// Warp-wide df64 sum (all lanes receive the result).
__device__ __forceinline__ f2 warp_sum_df(f2 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        f2 w{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
        v = df_add(v, w);
    }
    return v;
}

// Block-wide df64 sum returned as a df64 pair in every thread (converted to double where it is
// published, by one thread).
__device__ __forceinline__ f2 block_sum_df(f2 v)
{
    __shared__ f2 red_df[33];
    int t = threadIdx.x + threadIdx.y * blockDim.x;
    int nt = blockDim.x * blockDim.y;
    v = warp_sum_df(v);
    __syncthreads();
    if ((t & 31) == 0) red_df[t >> 5] = v;
    __syncthreads();
    if (t < 32) {
        f2 w = (t < (nt >> 5)) ? red_df[t] : f2{0.f, 0.f};
        w = warp_sum_df(w);
        if (t == 0) red_df[32] = w;
    }
    __syncthreads();
    const f2 r = red_df[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ float block_max_f(float v)
{
    __shared__ float red_mf[33];
    int t = threadIdx.x + threadIdx.y * blockDim.x;
    int nt = blockDim.x * blockDim.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((t & 31) == 0) red_mf[t >> 5] = v;
    __syncthreads();
    if (t < 32) {
        float w = (t < (nt >> 5)) ? red_mf[t] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w = fmaxf(w, __shfl_xor_sync(0xffffffffu, w, o));
        if (t == 0) red_mf[32] = w;
    }
    __syncthreads();
    float r = red_mf[32];
    __syncthreads();
    return r;
}

} // namespace envar
