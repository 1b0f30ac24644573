// plm_device.cuh -- small device helpers shared by the library's kernels:
// fixed-order (deterministic) block reductions in FP64, and double-float
// accumulation of FP32 products.
#pragma once
#include <cuda_runtime.h>

namespace plm {

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block in a fixed order; every thread gets the result.
// `red` must hold blockDim.x / 32 doubles; the call contains __syncthreads.
__device__ __forceinline__ double block_sum_d(double v, double *red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    v = warp_sum_d(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    for (int k = 0; k < nw; ++k) t += red[k];
    return t;
}

// Two sums at once (saves one barrier pair).
__device__ __forceinline__ void block_sum2_d(double &a, double &b, double *red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    __syncthreads();
    if (lane == 0) {
        red[2 * wid] = a;
        red[2 * wid + 1] = b;
    }
    __syncthreads();
    double ta = 0.0, tb = 0.0;
    for (int k = 0; k < nw; ++k) {
        ta += red[2 * k];
        tb += red[2 * k + 1];
    }
    a = ta;
    b = tb;
}

// Double-float accumulator (hi + lo, about 44 significant bits) of sums of
// FP32 products, in FP32 arithmetic (the FP64 pipe of this GPU is ~1/64 of
// FP32).  Terms enter through Knuth's two-sum, which adds them to (hi, lo)
// without rounding error, so the length of the sum adds no error.
//   df_fma  adds one product exactly: Dekker's two-product (the FMA gives
//           the rounding error of a*b), then the two-sum.
//   df_dot4 adds the four products of a float4 pair summed by an FMA chain:
//           its error is at most 4u of the sum of their magnitudes (u = 2^-24),
//           the order of the rounding already in the FP32 inputs, at a
//           quarter of df_fma's instructions per element.
// The _rn intrinsics keep the compiler from fusing or reassociating the
// error-free transformations.
struct DF {
    float hi = 0.0f, lo = 0.0f;
};

__device__ __forceinline__ void df_add(DF &s, float p)
{
    const float t = __fadd_rn(s.hi, p);
    const float bp = __fsub_rn(t, s.hi);
    const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s.hi = t;
    s.lo = __fadd_rn(s.lo, err);
}

__device__ __forceinline__ void df_fma(DF &s, float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);  // a*b - p, exact
    const float t = __fadd_rn(s.hi, p);
    const float bp = __fsub_rn(t, s.hi);
    const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s.hi = t;
    s.lo = __fadd_rn(s.lo, __fadd_rn(err, e));
}

__device__ __forceinline__ void df_dot4(DF &s, const float4 a, const float4 b)
{
    const float p = fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, __fmul_rn(a.x, b.x))));
    df_add(s, p);
}

__device__ __forceinline__ double df_value(const DF &s)
{
    return (double)s.hi + (double)s.lo;
}

}  // namespace plm
