// k_symmetric.cu -- the pieces symmetric plmDCA adds to the evaluation.
//
// Symmetric pseudolikelihood maximisation (Sec. 3, Eq. npll_1 with the l2
// penalty of Eq. l2reg) minimises l_pseudo + R_l2 with one coupling block
// per pair, J_ri = J_ir^T.  In the site-contiguous layout Theta[r][s][c]
// that is the sum over sites of the asymmetric objectives g_r^(reg) with
// lambda' = lambda_J / 2 (each block's penalty counted once from each of
// its two sites, the remark after Eq. g_reg), restricted to the subspace
// of layouts whose mirror blocks are transposes of each other.  The
// solver works in that subspace: its gradient is the orthogonal projection
// of the per-site gradient, G_ri <- (G_ri + G_ir^T) / 2, and its objective
// is the sum of the per-site data terms (the penalty is added by the
// line search from the trial point, as for the site problems).
#include "plm_device.cuh"
#include "plm_internal.cuh"

namespace plm {

namespace {

// block (i, j) = (blockIdx.y, blockIdx.x), i < j; thread (k, l)
__global__ void k_sym_project(float *__restrict__ G, Dims d)
{
    const int i = blockIdx.y, j = blockIdx.x;
    if (i >= j || (int)threadIdx.x >= Q * Q) return;
    const int k = threadIdx.x / Q, l = threadIdx.x % Q;
    float *a = G + ((size_t)i * QP + k) * d.KP + (size_t)j * Q + l;  // G_ij(k, l)
    float *b = G + ((size_t)j * QP + l) * d.KP + (size_t)i * Q + k;  // G_ji(l, k)
    const float m = 0.5f * (*a + *b);
    *a = m;
    *b = m;
}

// the sites' data terms summed in site order (one thread, FP64)
__global__ void k_sum_sites(const double *__restrict__ f, int n, double *out)
{
    double t = 0.0;
    for (int r = 0; r < n; ++r) t += f[r];
    *out = t;
}

}  // namespace

cudaError_t launch_sym_project(float *G, const Dims &d, cudaStream_t st)
{
    if (d.N > 1) {
        k_sym_project<<<dim3(d.N, d.N), (Q * Q + 31) / 32 * 32, 0, st>>>(G, d);
        count_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_sum_sites(const double *f, int n, double *out, cudaStream_t st)
{
    k_sum_sites<<<1, 1, 0, st>>>(f, n, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace plm
