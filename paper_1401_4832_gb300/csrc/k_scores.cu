// k_scores.cu -- steps 4-6 of the rundown: Ising gauge (Eq. gauge_change2),
// combination of the two estimates (Eq. average2, or the min/max
// alternatives of Sec. 6), Frobenius norm (Eq. frob_normtrans2), average
// product correction (Eq. corr_norm2) and the top-L contact list.
//
// For a pair i<j, site i's estimate is the block A(k,l) = J[i][k][j][l] and
// site j's estimate of the same coupling is J^j_ij(k,l) = J^j_ji(l,k) =
// J[j][l][i][k], i.e. the transpose of site j's stored block.  One warp
// handles one pair: both blocks are staged in shared memory in FP64, moved
// to the Ising gauge, combined elementwise and reduced to the pair's score:
// the Frobenius norm, or one of the Sec. 6 alternatives -- the general l_p
// norm, Burkoff's D_ij (Eqs. burkoffscore1-2), either norm without the gap
// state -- and the correction is the APC or the average sum correction
// (Eq. corr_normsum).
#include "plm_device.cuh"
#include "plm_internal.cuh"

namespace plm {

namespace {

constexpr int FN_WARPS = 4;

__global__ void __launch_bounds__(32 * FN_WARPS)
k_fn(const float *__restrict__ J, int N, int combine, ScoreKind sk, double *__restrict__ fn)
{
    __shared__ double A[FN_WARPS][Q][Q + 1];
    __shared__ double Bt[FN_WARPS][Q][Q + 1];
    __shared__ double mA[FN_WARPS][2][Q], mB[FN_WARPS][2][Q];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // block (x, y): row i = y, pairs (i, j) for j = x FN_WARPS + w; every
    // pair has its own warp
    const int i = blockIdx.y;
    const size_t NQ = (size_t)N * Q;
    if (lane == 0 && w == 0 && blockIdx.x == 0) fn[(size_t)i * N + i] = 0.0;
    {
        const int j = blockIdx.x * FN_WARPS + w;
        if (j <= i || j >= N) return;
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
        if (combine == 0) {
            // mean of the two estimates: the Ising gauge is linear, so the
            // mean is formed first and gauged once, C = (A + B^T) / 2
            double rowC = 0.0;
            if (lane < Q)
                for (int l = 0; l < Q; ++l) {
                    const double c = 0.5 * (A[w][lane][l] + Bt[w][lane][l]);
                    Bt[w][lane][l] = c;
                    rowC += c;
                }
            __syncwarp();
            double colC = 0.0;
            if (lane < Q) {
                for (int k = 0; k < Q; ++k) colC += Bt[w][k][lane];
                rowC /= Q;
                colC /= Q;
                mA[w][0][lane] = rowC;
                mA[w][1][lane] = colC;
            }
            const double allC = warp_sum_d(lane < Q ? rowC : 0.0) / Q;
            __syncwarp();
            if (lane < Q)
                for (int l = 0; l < Q; ++l)
                    Bt[w][lane][l] = Bt[w][lane][l] - mA[w][1][l] - mA[w][0][lane] + allC;
        } else {
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
            // the combined gauged block (min or max of the two gauged
            // estimates), row k = lane
            if (lane < Q) {
                const int k = lane;
                for (int l = 0; l < Q; ++l) {
                    double a = A[w][k][l] - mA[w][1][l] - mA[w][0][k] + allA;
                    double b = Bt[w][k][l] - mB[w][1][l] - mB[w][0][k] + allB;
                    Bt[w][k][l] = combine == 1 ? fmin(a, b) : fmax(a, b);
                }
            }
        }
        __syncwarp();
        double out;
        if (sk.kind == 2) {
            // Burkoff: P = f_i(k) f_j(l) e^(v - vmax) / Z and ln(P / (f_i f_j))
            // = v - vmax - ln Z; the block maximum vmax cancels in P and keeps
            // every exponential finite
            const double *fi = sk.freq + (size_t)i * Q, *fj = sk.freq + (size_t)j * Q;
            double vmax = -INFINITY;
            if (lane < Q)
                for (int l = 0; l < Q; ++l) vmax = fmax(vmax, Bt[w][lane][l]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
            // the unnormalised weights f_i f_j e^(v - vmax), kept in A (free
            // after the gauge) for the second pass
            double z = 0.0;
            if (lane < Q)
                for (int l = 0; l < Q; ++l) {
                    const double u = fi[lane] * fj[l] * exp(Bt[w][lane][l] - vmax);
                    A[w][lane][l] = u;
                    z += u;
                }
            const double Z = warp_sum_d(z);
            const double lz = log(Z) + vmax;
            double d = 0.0;
            if (lane < Q)
                for (int l = 0; l < Q; ++l) {
                    const double P = A[w][lane][l] / Z;
                    if (P > 0.0) d += P * (Bt[w][lane][l] - lz);
                }
            out = warp_sum_d(d);
        } else {
            // l_p with p = 1 is the sum of |a| and with p = 2 the Frobenius
            // norm: no pow for those (pow(a, 1) = a exactly)
            const int pk = sk.kind != 1 ? 2 : sk.p == 1.0 ? 1 : sk.p == 2.0 ? 2 : 0;
            double ss = 0.0;
            if (lane < Q && !(sk.exclude_gap && lane == 0))
                for (int l = sk.exclude_gap ? 1 : 0; l < Q; ++l) {
                    const double a = fabs(Bt[w][lane][l]);
                    ss += pk == 1 ? a : pk == 2 ? a * a : pow(a, sk.p);
                }
            ss = warp_sum_d(ss);
            out = pk == 1 ? ss : pk == 2 ? sqrt(ss) : pow(ss, 1.0 / sk.p);
        }
        if (lane == 0) {
            fn[(size_t)i * N + j] = out;
            fn[(size_t)j * N + i] = out;
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

// one warp: the grand total of the raw row sums (lanes take alternate rows,
// then a fixed-order butterfly), the row means and the total mean
__global__ void k_apc_total(double *__restrict__ row, int N)
{
    const int lane = threadIdx.x & 31;
    double tot = 0.0;
    for (int i = lane; i < N; i += 32) tot += row[i];
    tot = warp_sum_d(tot);
    __syncwarp();
    for (int i = lane; i < N; i += 32) row[i] /= (N - 1);
    if (lane == 0) row[N] = tot / ((double)N * (N - 1));
}

// correction 0: APC (Eq. corr_norm2); 1: average sum correction (Eq.
// corr_normsum); 2: none
__global__ void k_apc_apply(const double *__restrict__ fn, int N,
                            const double *__restrict__ row,
                            double *__restrict__ cfn, int correction)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)N * N) return;
    int i = (int)(idx / N), j = (int)(idx % N);
    double tot = row[N];
    double c;
    if (correction == 1) c = row[j] + row[i] - tot;
    else if (correction == 2) c = 0.0;
    else c = tot > 0.0 ? row[j] * row[i] / tot : 0.0;  // all-zero FN: 0/0 taken as 0
    cfn[idx] = (i == j) ? 0.0 : fn[idx] - c;
}

// f[i][k] = (1/B_eff) sum_b w_b [S_bi = k]: one block per position, a fixed
// order of partial sums
__global__ void k_site_freqs(const int8_t *__restrict__ msa, const float *__restrict__ w, int B,
                             int N, double inv_beff, double *__restrict__ f)
{
    __shared__ double part[128][Q + 1];
    const int i = blockIdx.x, t = threadIdx.x;
    double acc[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) acc[k] = 0.0;
    for (int b = t; b < B; b += 128) {
        const int s = msa[(size_t)b * N + i];
        const double wb = w[b];
#pragma unroll
        for (int k = 0; k < Q; ++k) acc[k] += (s == k) ? wb : 0.0;
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) part[t][k] = acc[k];
    __syncthreads();
    if (t < Q) {
        double s = 0.0;
        for (int u = 0; u < 128; ++u) s += part[u][t];
        f[(size_t)i * Q + t] = s * inv_beff;
    }
}

// ---- top-L selection ----------------------------------------------------
// Order: score descending, then (i, j) ascending.  Each eligible pair gets a
// 96-bit composite key (hi: the score's bits mapped to an order-preserving
// unsigned integer; lo: 0xFFFFFFFF - (i N + j)), unique per pair, larger =
// earlier.  A most-significant-byte-first radix select finds the L-th
// largest key in 12 histogram passes; the pairs at or above it (exactly L)
// are gathered and sorted by one CTA (bitonic sort).

struct SelState {
    unsigned long long pre_hi;  // determined high part of the L-th key
    unsigned int pre_lo;
    unsigned int k;             // rank still to find inside the current prefix
    unsigned int count;         // gathered candidates
    unsigned int eligible;
    unsigned int done;          // the prefix already selects exactly the top k
    unsigned int hist[256];
};

__device__ __forceinline__ unsigned long long score_key(double v)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ bool eligible(long long idx, int N, int min_sep)
{
    const int i = (int)(idx / N), j = (int)(idx % N);
    return j - i >= min_sep;
}

// byte t (0 = most significant) of the composite key
__device__ __forceinline__ unsigned int key_byte(unsigned long long hi, unsigned int lo, int t)
{
    return t < 8 ? (unsigned int)(hi >> (56 - 8 * t)) & 0xFFu
                 : (lo >> (24 - 8 * (t - 8))) & 0xFFu;
}

// does the key agree with the prefix on bytes 0..t-1?
__device__ __forceinline__ bool prefix_match(unsigned long long hi, unsigned int lo,
                                             const SelState *st, int t)
{
    if (t == 0) return true;
    if (t <= 8) {
        const int sh = 64 - 8 * t;
        return (hi >> sh) == (st->pre_hi >> sh);
    }
    if (hi != st->pre_hi) return false;
    const int sh = 32 - 8 * (t - 8);
    return (lo >> sh) == (st->pre_lo >> sh);
}

__global__ void k_sel_init(SelState *st, const double *score, int N, int L, int min_sep)
{
    // one block: count eligible pairs
    __shared__ unsigned int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    unsigned int c = 0;
    for (long long idx = threadIdx.x; idx < (long long)N * N; idx += blockDim.x)
        if (eligible(idx, N, min_sep)) c++;
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) {
        st->eligible = cnt;
        st->k = (unsigned int)min((unsigned int)L, cnt);
        st->pre_hi = 0;
        st->pre_lo = 0;
        st->count = 0;
        st->done = 0;
    }
    for (int b = threadIdx.x; b < 256; b += blockDim.x) st->hist[b] = 0;
}

__global__ void k_sel_hist(SelState *st, const double *__restrict__ score, int N, int min_sep,
                           int t)
{
    if (st->done) return;  // the remaining passes have nothing to decide
    __shared__ unsigned int h[256];
    for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const long long total = (long long)N * N;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        if (!eligible(idx, N, min_sep)) continue;
        const unsigned long long hi = score_key(score[idx]);
        const unsigned int lo = 0xFFFFFFFFu - (unsigned int)idx;
        if (prefix_match(hi, lo, st, t)) atomicAdd(&h[key_byte(hi, lo, t)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (h[b]) atomicAdd(&st->hist[b], h[b]);
}

// One warp: the digit of byte t of the k-th largest key among those that
// match the prefix (lane l scans bins 255 - 8l down to 248 - 8l, an
// exclusive scan over the lanes orders the lanes' totals from the top).
// When every key in the chosen bin is among the top k (the bin's count is
// exactly the rank still to find), the prefix with zero lower bytes
// already separates the top k from the rest: the remaining passes are
// skipped and the gather takes the same set.
__global__ void k_sel_pick(SelState *st, int t)
{
    const int lane = threadIdx.x & 31;
    if (st->k == 0 || st->done) return;  // nothing to select (the histogram is empty)
    const unsigned int k = st->k;
    unsigned int c[8], sum = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        c[u] = st->hist[255 - 8 * lane - u];
        sum += c[u];
    }
    unsigned int pre = sum;  // inclusive scan over the lanes, then made exclusive
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int v = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += v;
    }
    pre -= sum;
    const unsigned int mine = __ballot_sync(0xffffffffu, pre < k && k <= pre + sum);
    if (lane == __ffs(mine) - 1) {
        unsigned int acc = pre;
        int digit = 0;
        unsigned int cnt = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (acc + c[u] >= k) {
                digit = 255 - 8 * lane - u;
                cnt = c[u];
                break;
            }
            acc += c[u];
        }
        st->k = k - acc;
        if (t < 8) st->pre_hi |= (unsigned long long)digit << (56 - 8 * t);
        else st->pre_lo |= (unsigned int)digit << (24 - 8 * (t - 8));
        if (acc + cnt == k) st->done = 1;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) st->hist[255 - 8 * lane - u] = 0;
}

struct Cand {
    unsigned long long hi;
    unsigned int lo;
    unsigned int pad;
};

__device__ __forceinline__ bool cand_before(const Cand &a, const Cand &b)
{
    return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}

__global__ void k_sel_gather(SelState *st, const double *__restrict__ score, int N, int min_sep,
                             Cand *cand, int L)
{
    if (st->k == 0 && st->eligible == 0) return;
    const long long total = (long long)N * N;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        if (!eligible(idx, N, min_sep)) continue;
        const unsigned long long hi = score_key(score[idx]);
        const unsigned int lo = 0xFFFFFFFFu - (unsigned int)idx;
        const bool ge = hi > st->pre_hi || (hi == st->pre_hi && lo >= st->pre_lo);
        if (st->eligible <= (unsigned int)L || ge) {
            const unsigned int pos = atomicAdd(&st->count, 1u);
            if (pos < (unsigned int)L) cand[pos] = Cand{hi, lo, 0};
        }
    }
}

// one CTA: bitonic sort of the gathered candidates (power-of-two padded)
__global__ void k_sel_sort(const SelState *st, Cand *cand, int n2, int L, int N, int32_t *ij)
{
    extern __shared__ Cand sh[];
    const unsigned int n = min(st->count, (unsigned int)L);
    for (int t = threadIdx.x; t < n2; t += blockDim.x)
        sh[t] = (t < (int)n) ? cand[t] : Cand{0ull, 0u, 0u};
    __syncthreads();
    for (int size = 2; size <= n2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < n2; t += blockDim.x) {
                const int partner = t ^ stride;
                if (partner > t) {
                    const bool desc = (t & size) == 0;
                    const bool swap = desc ? cand_before(sh[partner], sh[t])
                                           : cand_before(sh[t], sh[partner]);
                    if (swap) {
                        const Cand tmp = sh[t];
                        sh[t] = sh[partner];
                        sh[partner] = tmp;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < L; t += blockDim.x) {
        if (t < (int)n) {
            const unsigned int idx = 0xFFFFFFFFu - sh[t].lo;
            ij[2 * t] = (int32_t)(idx / N);
            ij[2 * t + 1] = (int32_t)(idx % N);
        } else {
            ij[2 * t] = -1;
            ij[2 * t + 1] = -1;
        }
    }
}

}  // namespace

cudaError_t launch_fn(const float *J, int N, int combine, double *fn,
                      cudaStream_t st, ScoreKind sk)
{
    k_fn<<<dim3((N + FN_WARPS - 1) / FN_WARPS, N), 32 * FN_WARPS, 0, st>>>(J, N, combine, sk, fn);
    count_launches(1);
    return cudaGetLastError();
}

// work: N + 1 doubles
cudaError_t launch_apc(const double *fn, int N, double *cfn, double *work,
                       cudaStream_t st, int correction)
{
    k_apc_rows<<<(N + 127) / 128, 128, 0, st>>>(fn, N, work);
    k_apc_total<<<1, 32, 0, st>>>(work, N);
    size_t nn = (size_t)N * N;
    k_apc_apply<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(fn, N, work, cfn, correction);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_site_freqs(const int8_t *msa, const float *w, int B, int N, double beff,
                              double *f, cudaStream_t st)
{
    k_site_freqs<<<N, 128, 0, st>>>(msa, w, B, N, 1.0 / beff, f);
    count_launches(1);
    return cudaGetLastError();
}

constexpr int TOPL_MAX = 8192;  // largest L sorted in one CTA

size_t topL_scratch_bytes(int L)
{
    return sizeof(SelState) + 256 + (size_t)(L > 0 ? L : 1) * sizeof(Cand);
}

cudaError_t launch_topL(const double *score, int N, int L, int min_sep, int32_t *ij,
                        void *scratch, cudaStream_t st)
{
    if (L <= 0) return cudaSuccess;
    if (L > TOPL_MAX || (long long)N * N >= 0xFFFFFFFFll) return cudaErrorInvalidValue;
    static std::atomic<unsigned long long> attr{0};
    cudaError_t e = set_smem_limit_once((const void *)k_sel_sort, TOPL_MAX * (int)sizeof(Cand),
                                        attr);
    if (e) return e;
    SelState *ss = (SelState *)scratch;
    Cand *cand = (Cand *)((char *)scratch + ((sizeof(SelState) + 255) / 256) * 256);
    k_sel_init<<<1, 256, 0, st>>>(ss, score, N, L, min_sep);
    const long long total = (long long)N * N;
    const int grid = (int)min((total + 255) / 256, 4LL * 152);
    for (int t = 0; t < 12; ++t) {
        k_sel_hist<<<grid, 256, 0, st>>>(ss, score, N, min_sep, t);
        k_sel_pick<<<1, 32, 0, st>>>(ss, t);
    }
    k_sel_gather<<<grid, 256, 0, st>>>(ss, score, N, min_sep, cand, L);
    int n2 = 1;
    while (n2 < L) n2 <<= 1;
    k_sel_sort<<<1, 1024, (size_t)n2 * sizeof(Cand), st>>>(ss, cand, n2, L, N, ij);
    count_launches(1 + 2 * 12 + 2);
    return cudaGetLastError();
}

}  // namespace plm
