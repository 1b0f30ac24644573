// k_layout.cu -- conversion between the public (h, J) layout and the padded
// site-contiguous Theta layout, and the per-site l2 penalty of Eq. g_regdef2.
#include "plm_device.cuh"
#include "plm_internal.cuh"

namespace plm {

namespace {

__global__ void k_pack_theta(const float *__restrict__ h,
                             const float *__restrict__ J, Dims d,
                             float *__restrict__ theta)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = d.theta_elems();
    if (idx >= total) return;
    int c = (int)(idx % d.KP);
    int row = (int)(idx / d.KP);
    int r = row / QP, s = row % QP;
    float v = 0.0f;
    const int NQ = d.N * Q;
    if (s < Q) {
        if (c < NQ) {
            int i = c / Q;
            if (i != r) v = J[((size_t)r * Q + s) * NQ + c];
        } else if (c == NQ) {
            v = h[(size_t)r * Q + s];
        }
    }
    theta[idx] = v;
}

__global__ void k_unpack_theta(const float *__restrict__ theta, Dims d,
                               float *__restrict__ h, float *__restrict__ J)
{
    const int NQ = d.N * Q;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)d.N * Q * (NQ + 1);
    if (idx >= total) return;
    int c = (int)(idx % (NQ + 1));
    size_t rs = idx / (NQ + 1);
    int r = (int)(rs / Q), s = (int)(rs % Q);
    float v = theta[((size_t)r * QP + s) * d.KP + c];
    if (c < NQ) {
        if (J) J[rs * NQ + c] = (c / Q == r) ? 0.0f : v;
    } else if (h) {
        h[rs] = v;
    }
}

// one block per site: lambda_h sum_s h_r(s)^2 + lambda'_J sum_{s, c<NQ} J^2
__global__ void __launch_bounds__(512)
k_penalty(const float *__restrict__ theta, Dims d, double lambda_h,
          double lambda_Jp, double *__restrict__ pen)
{
    __shared__ double red[64];
    const int r = blockIdx.x;
    const float *th = theta + (size_t)r * d.site_elems();
    const int NQ = d.N * Q;
    double sj = 0.0, sh = 0.0;
    for (int s = 0; s < Q; ++s) {
        const float *row = th + (size_t)s * d.KP;
        for (int c = threadIdx.x; c <= NQ; c += blockDim.x) {
            double v = row[c];
            if (c < NQ) sj += v * v;
            else sh += v * v;
        }
    }
    block_sum2_d(sj, sh, red);
    if (threadIdx.x == 0) pen[r] = lambda_h * sh + lambda_Jp * sj;
}

}  // namespace

cudaError_t launch_pack_theta(const float *h, const float *J, const Dims &d,
                              float *theta, cudaStream_t st)
{
    size_t total = d.theta_elems();
    k_pack_theta<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(h, J, d, theta);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_unpack_theta(const float *theta, const Dims &d, float *h,
                                float *J, cudaStream_t st)
{
    size_t total = (size_t)d.N * Q * (d.N * Q + 1);
    k_unpack_theta<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(theta, d, h, J);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_penalty(const float *theta, const Dims &d, double lambda_h,
                           double lambda_Jp, double *pen, cudaStream_t st)
{
    k_penalty<<<d.N, 512, 0, st>>>(theta, d, lambda_h, lambda_Jp, pen);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace plm
