// k_tc.cu -- split-BF16 tensor-core (tcgen05) path: placeholder until the
// contraction kernels land; only the theta split is implemented.
#include "plm_internal.cuh"

namespace plm {

namespace {
__global__ void k_split(const float *__restrict__ theta, size_t n,
                        __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    float x = theta[idx];
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[idx] = h;
    lo[idx] = __float2bfloat16_rn(x - __bfloat162float(h));
}
}  // namespace

cudaError_t launch_split_theta(const float *theta, const Dims &d,
                               __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                               cudaStream_t st)
{
    size_t n = d.theta_elems();
    k_split<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(theta, n, hi, lo);
    count_launches(1);
    return cudaGetLastError();
}

size_t tc_scratch_bytes(const Dims &) { return 256; }
int tc_supported() { return 0; }

cudaError_t launch_tc_eval(void *, const int8_t *, const float *, double,
                           const __nv_bfloat16 *, const __nv_bfloat16 *,
                           const float *, const Dims &, double, double, void *,
                           double *, float *, int *, cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace plm
