// plm_device.cuh -- small device helpers shared by the library's kernels:
// fixed-order (deterministic) block reductions in FP64.
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

}  // namespace plm
