// k_scores.cu -- steps 4-6 of the rundown: Ising gauge (Eq. gauge_change2),
// combination of the two estimates (Eq. average2, or the min/max
// alternatives of Sec. 6), Frobenius norm (Eq. frob_normtrans2), average
// product correction (Eq. corr_norm2) and the top-L contact list.
//
// For a pair i<j, site i's estimate is the block A(k,l) = J[i][k][j][l] and
// site j's estimate of the same coupling is J^j_ij(k,l) = J^j_ji(l,k) =
// J[j][l][i][k], i.e. the transpose of site j's stored block.  One warp
// handles one pair: both blocks are staged in shared memory in FP64, moved
// to the Ising gauge, combined elementwise and reduced to the norm.
#include "plm_device.cuh"
#include "plm_internal.cuh"

namespace plm {

namespace {

constexpr int FN_WARPS = 4;

__global__ void __launch_bounds__(32 * FN_WARPS)
k_fn(const float *__restrict__ J, int N, int combine, double *__restrict__ fn)
{
    __shared__ double A[FN_WARPS][Q][Q + 1];
    __shared__ double Bt[FN_WARPS][Q][Q + 1];
    __shared__ double mA[FN_WARPS][2][Q], mB[FN_WARPS][2][Q];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x;
    const size_t NQ = (size_t)N * Q;
    if (lane == 0 && w == 0) fn[(size_t)i * N + i] = 0.0;
    for (int j = i + 1 + w; j < N; j += FN_WARPS) {
        if (lane < Q) {
            const float *ra = J + ((size_t)i * Q + lane) * NQ + (size_t)j * Q;  // J[i][lane][j][.]
            const float *rb = J + ((size_t)j * Q + lane) * NQ + (size_t)i * Q;  // J[j][lane][i][.]
#pragma unroll
            for (int l = 0; l < Q; ++l) {
                A[w][lane][l] = ra[l];
                Bt[w][l][lane] = rb[l];  // transpose: Bt(k,l) = J[j][l][i][k]
            }
        }
        __syncwarp();
        double rowA = 0, colA = 0, rowB = 0, colB = 0;
        if (lane < Q) {
            for (int l = 0; l < Q; ++l) {
                rowA += A[w][lane][l];
                colA += A[w][l][lane];
                rowB += Bt[w][lane][l];
                colB += Bt[w][l][lane];
            }
            rowA /= Q; colA /= Q; rowB /= Q; colB /= Q;
            mA[w][0][lane] = rowA; mA[w][1][lane] = colA;
            mB[w][0][lane] = rowB; mB[w][1][lane] = colB;
        }
        double allA = warp_sum_d(lane < Q ? rowA : 0.0) / Q;
        double allB = warp_sum_d(lane < Q ? rowB : 0.0) / Q;
        __syncwarp();
        double ss = 0.0;
        if (lane < Q) {
            const int k = lane;
            for (int l = 0; l < Q; ++l) {
                double a = A[w][k][l] - mA[w][1][l] - mA[w][0][k] + allA;
                double b = Bt[w][k][l] - mB[w][1][l] - mB[w][0][k] + allB;
                double v = combine == 1 ? fmin(a, b) : combine == 2 ? fmax(a, b) : 0.5 * (a + b);
                ss += v * v;
            }
        }
        ss = warp_sum_d(ss);
        if (lane == 0) {
            double v = sqrt(ss);
            fn[(size_t)i * N + j] = v;
            fn[(size_t)j * N + i] = v;
        }
        __syncwarp();
    }
}

// row[i] = sum_{j != i} fn[i][j] / (N-1); work[N] = total mean
__global__ void k_apc_rows(const double *__restrict__ fn, int N,
                           double *__restrict__ row)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = 0.0;
    for (int j = 0; j < N; ++j)
        if (j != i) s += fn[(size_t)i * N + j];
    row[i] = s;  // the raw sum; divided below
}

__global__ void k_apc_total(double *__restrict__ row, int N)
{
    if (threadIdx.x != 0) return;
    double tot = 0.0;
    for (int i = 0; i < N; ++i) tot += row[i];
    for (int i = 0; i < N; ++i) row[i] /= (N - 1);
    row[N] = tot / ((double)N * (N - 1));
}

__global__ void k_apc_apply(const double *__restrict__ fn, int N,
                            const double *__restrict__ row,
                            double *__restrict__ cfn)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)N * N) return;
    int i = (int)(idx / N), j = (int)(idx % N);
    double tot = row[N];
    // all-zero FN makes the correction 0/0; it is taken as 0
    cfn[idx] = (i == j) ? 0.0 : fn[idx] - (tot > 0.0 ? row[j] * row[i] / tot : 0.0);
}

// rank of pair (i,j) = number of eligible pairs ordered before it
// (score descending, then i ascending, then j ascending)
constexpr int TL_CHUNK = 1024;

__global__ void __launch_bounds__(256)
k_topL(const double *__restrict__ score, int N, int L, int min_sep,
       int32_t *__restrict__ ij)
{
    __shared__ double cs[TL_CHUNK];
    __shared__ int ci[TL_CHUNK];
    const long long total = (long long)N * N;
    long long me = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int mi = (int)(me / N), mj = (int)(me % N);
    const bool valid = me < total && mj - mi >= min_sep;
    const double ms = valid ? score[me] : 0.0;
    long long rank = 0;
    for (long long c0 = 0; c0 < total; c0 += TL_CHUNK) {
        __syncthreads();
        for (int t = threadIdx.x; t < TL_CHUNK; t += blockDim.x) {
            long long o = c0 + t;
            int oi = (int)(o / N), oj = (int)(o % N);
            bool ok = o < total && oj - oi >= min_sep;
            cs[t] = ok ? score[o] : 0.0;
            ci[t] = ok ? 1 : 0;
        }
        __syncthreads();
        if (valid) {
            for (int t = 0; t < TL_CHUNK; ++t) {
                if (!ci[t]) continue;
                long long o = c0 + t;
                double v = cs[t];
                // row-major index order equals (i, j) ascending
                if (v > ms || (v == ms && o < me)) rank++;
            }
        }
    }
    if (valid && rank < L) {
        ij[2 * rank] = mi;
        ij[2 * rank + 1] = mj;
    }
}

__global__ void k_fill_i32(int32_t *p, size_t n, int32_t v)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) p[idx] = v;
}

}  // namespace

cudaError_t launch_fn(const float *J, int N, int combine, double *fn,
                      cudaStream_t st)
{
    k_fn<<<N, 32 * FN_WARPS, 0, st>>>(J, N, combine, fn);
    count_launches(1);
    return cudaGetLastError();
}

// work: N + 1 doubles
cudaError_t launch_apc(const double *fn, int N, double *cfn, double *work,
                       cudaStream_t st)
{
    k_apc_rows<<<(N + 127) / 128, 128, 0, st>>>(fn, N, work);
    k_apc_total<<<1, 32, 0, st>>>(work, N);
    size_t nn = (size_t)N * N;
    k_apc_apply<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(fn, N, work, cfn);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_topL(const double *score, int N, int L, int min_sep,
                        int32_t *ij, cudaStream_t st)
{
    if (L <= 0) return cudaSuccess;
    size_t n = 2 * (size_t)L;
    k_fill_i32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ij, n, -1);
    size_t total = (size_t)N * N;
    k_topL<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(score, N, L, min_sep, ij);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace plm
