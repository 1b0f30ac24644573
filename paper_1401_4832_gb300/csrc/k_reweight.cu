// k_reweight.cu -- sequence reweighting, step 2 of the rundown (Eq.
// inverse_weights2; Sec. 3.1, Eq. inverse_weights).
//
// Sequences are packed into 5 bit-planes (states 0..20 fit in 5 bits): bit j
// of word w of plane p is bit p of S[b][32w + j].  Two sequences differ at a
// position iff some plane differs there, so
//     mismatches(a,b) = sum_w popc( OR_p (P_p[a][w] ^ P_p[b][w]) )
// and they are similar iff N - mismatches >= T = ceil(x N).  Padding bits
// beyond N are zero in every plane, so they never count as mismatches.
// Only tiles on or above the diagonal are visited; an off-diagonal tile adds
// its row counts to m[a] and its column counts to m[b].  All counts are
// integers, so the result does not depend on the order of the atomics.
#include "plm_internal.cuh"

namespace plm {

namespace {

constexpr int RW_TILE = 64;   // sequences per tile side
constexpr int RW_WC = 16;     // words per staged chunk

__global__ void k_pack_planes(const int8_t *__restrict__ msa, int B, int N,
                              int W, uint32_t *__restrict__ planes,
                              int *__restrict__ err)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)B * W) return;
    int b = (int)(idx / W), w = (int)(idx % W);
    uint32_t p[5] = {0, 0, 0, 0, 0};
    int bad = 0;
    for (int j = 0; j < 32; ++j) {
        int i = w * 32 + j;
        if (i >= N) break;
        int s = msa[(size_t)b * N + i];
        if (s < 0 || s >= Q) bad = 1;
#pragma unroll
        for (int t = 0; t < 5; ++t) p[t] |= (uint32_t)((s >> t) & 1) << j;
    }
    if (bad) atomicOr(err, 1);
#pragma unroll
    for (int t = 0; t < 5; ++t) planes[((size_t)t * B + b) * W + w] = p[t];
}

__global__ void __launch_bounds__(256)
k_pair_counts(const uint32_t *__restrict__ planes, int B, int N, int W,
              int max_mism, int32_t *__restrict__ m)
{
    const int ta = blockIdx.y, tb = blockIdx.x;
    if (ta > tb) return;
    __shared__ uint32_t sa[5][RW_WC][RW_TILE];
    __shared__ uint32_t sb[5][RW_WC][RW_TILE];
    __shared__ int rowc[RW_TILE], colc[RW_TILE];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int a0 = ta * RW_TILE, b0 = tb * RW_TILE;
    if (tid < RW_TILE) {
        rowc[tid] = 0;
        colc[tid] = 0;
    }
    int mism[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) mism[u][v] = 0;

    for (int w0 = 0; w0 < W; w0 += RW_WC) {
        __syncthreads();
        // stage 5 planes x RW_WC words x 64 rows for both tiles
        for (int e = tid; e < 5 * RW_WC * RW_TILE; e += blockDim.x) {
            int row = e % RW_TILE;
            int ww = (e / RW_TILE) % RW_WC;
            int p = e / (RW_TILE * RW_WC);
            int w = w0 + ww;
            uint32_t va = 0, vb = 0;
            if (w < W) {
                if (a0 + row < B) va = planes[((size_t)p * B + a0 + row) * W + w];
                if (b0 + row < B) vb = planes[((size_t)p * B + b0 + row) * W + w];
            }
            sa[p][ww][row] = va;
            sb[p][ww][row] = vb;
        }
        __syncthreads();
        const int wn = min(RW_WC, W - w0);
        for (int ww = 0; ww < wn; ++ww) {
            uint32_t A[5][4], Bv[5][4];
#pragma unroll
            for (int p = 0; p < 5; ++p)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    A[p][u] = sa[p][ww][ty * 4 + u];
                    Bv[p][u] = sb[p][ww][tx * 4 + u];
                }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    uint32_t x = (A[0][u] ^ Bv[0][v]) | (A[1][u] ^ Bv[1][v]) |
                                 (A[2][u] ^ Bv[2][v]) | (A[3][u] ^ Bv[3][v]) |
                                 (A[4][u] ^ Bv[4][v]);
                    mism[u][v] += __popc(x);
                }
        }
    }
    // similar iff matches >= T  <=>  mismatches <= N - T
    int rsum[4] = {0, 0, 0, 0}, csum[4] = {0, 0, 0, 0};
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int a = a0 + ty * 4 + u, b = b0 + tx * 4 + v;
            int sim = (a < B && b < B && mism[u][v] <= max_mism) ? 1 : 0;
            rsum[u] += sim;
            csum[v] += sim;
        }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        if (rsum[u]) atomicAdd(&rowc[ty * 4 + u], rsum[u]);
        if (csum[u]) atomicAdd(&colc[tx * 4 + u], csum[u]);
    }
    __syncthreads();
    if (tid < RW_TILE) {
        // column counts: m[b] += #{a in tile a : similar}
        if (b0 + tid < B && colc[tid]) atomicAdd(&m[b0 + tid], colc[tid]);
        // row counts only off the diagonal (the mirror tile is not visited)
        if (ta != tb && a0 + tid < B && rowc[tid]) atomicAdd(&m[a0 + tid], rowc[tid]);
    }
}

__global__ void k_weights(const int32_t *__restrict__ m, int B,
                          float *__restrict__ w, int32_t *__restrict__ hist)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    int mb = m[b];
    if (w) w[b] = 1.0f / (float)mb;  // IEEE round-to-nearest division
    atomicAdd(&hist[mb], 1);
}

// B_eff = sum_{k=1..B} hist[k] / k, added in increasing k by one lane so that
// the rounding sequence is fixed; chunks of 32 empty bins are skipped.
__global__ void k_beff(const int32_t *__restrict__ hist, int B,
                       double *__restrict__ beff)
{
    const int lane = threadIdx.x;
    double acc = 0.0;
    for (int k0 = 1; k0 <= B; k0 += 32) {
        int k = k0 + lane;
        int hk = (k <= B) ? hist[k] : 0;
        unsigned nz = __ballot_sync(0xffffffffu, hk != 0);
        if (!nz) continue;
        double term = hk ? (double)hk / (double)k : 0.0;
        for (int j = 0; j < 32; ++j) {
            double t = __shfl_sync(0xffffffffu, term, j);
            if ((nz >> j) & 1u) acc += t;
        }
    }
    if (lane == 0) *beff = acc;
}

}  // namespace

size_t reweight_scratch_bytes(int B, int N)
{
    size_t W = ((size_t)N + 31) / 32;
    size_t planes = 5 * (size_t)B * W * sizeof(uint32_t);
    planes = (planes + 255) / 256 * 256;
    size_t m = ((size_t)B * sizeof(int32_t) + 255) / 256 * 256;
    size_t hist = (((size_t)B + 1) * sizeof(int32_t) + 255) / 256 * 256;
    return planes + m + hist;
}

// scratch layout: planes | m (used when m_out is NULL) | hist
cudaError_t launch_reweight(const int8_t *msa, int B, int N, int T,
                            int32_t *m_out, float *w_out, double *beff_dev,
                            void *scratch, int *err, cudaStream_t st)
{
    const int W = (N + 31) / 32;
    char *p = (char *)scratch;
    uint32_t *planes = (uint32_t *)p;
    size_t planes_b = (5 * (size_t)B * W * sizeof(uint32_t) + 255) / 256 * 256;
    int32_t *m_tmp = (int32_t *)(p + planes_b);
    size_t m_b = ((size_t)B * sizeof(int32_t) + 255) / 256 * 256;
    int32_t *hist = (int32_t *)(p + planes_b + m_b);
    int32_t *m = m_out ? m_out : m_tmp;

    cudaError_t e;
    if ((e = cudaMemsetAsync(m, 0, (size_t)B * sizeof(int32_t), st))) return e;
    if ((e = cudaMemsetAsync(hist, 0, ((size_t)B + 1) * sizeof(int32_t), st))) return e;
    size_t nw = (size_t)B * W;
    k_pack_planes<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(msa, B, N, W, planes, err);
    int tiles = (B + RW_TILE - 1) / RW_TILE;
    dim3 grid(tiles, tiles);
    k_pair_counts<<<grid, 256, 0, st>>>(planes, B, N, W, N - T, m);
    k_weights<<<(B + 255) / 256, 256, 0, st>>>(m, B, w_out, hist);
    k_beff<<<1, 32, 0, st>>>(hist, B, beff_dev);
    count_launches(4);
    return cudaGetLastError();
}

}  // namespace plm
