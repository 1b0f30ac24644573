// k_gather.cu -- the exact-FP32 objective/gradient path on the CUDA cores.
//
// Logits (Eq. condpfinal):  L[b][(r,s)] = sum_i Theta[(r,s)][i*Q + S_bi] + h_r(s)
// i.e. the one-hot product X Theta^T done as gathers: for every position i
// only the column of the observed state contributes.  A CTA stages a tile
// of 128 rows (r,s) x 4 positions x 21 states of Theta transposed in shared
// memory (row stride 129 words, so both the staging stores and the lane-wise
// loads are bank-conflict free; two chunks in flight, staged by cp.async) and
// each warp sums the gathered entries for 16 sequences.
//
// Log-softmax, objective and residual (Eq. g_regdef2; Eqs. g_gradh2,
// g_gradJ2): one thread per (site, sequence) over the 21 states in FP32,
// objective partial sums in FP64 in a fixed order.
//
// Gradient (Eq. g_gradJ2):  G[(r,s)][i*Q + k] = sum_b D[b][(r,s)] [S_bi == k]
// A CTA owns 128 rows x 8 positions (one position per warp); each lane keeps
// 21 x 4 accumulators in registers.  Residual tiles of 32 sequences are
// staged by cp.async into two shared buffers; for each state k the warp
// takes the mask of the tile's sequences showing k at its position (a
// ballot, the same for all lanes) and adds their residual rows to the
// state's accumulators in sequence order.
#include "plm_device.cuh"
#include "plm_internal.cuh"

namespace plm {

namespace {

constexpr int LG_ROWS = 128;        // rows (r,s) per CTA
constexpr int LG_IC = 4;            // positions per staged chunk (two chunks in flight)
constexpr int LG_BPW = 16;          // sequences per warp
constexpr int LG_BT = 8 * LG_BPW;   // sequences per CTA
constexpr int LG_STRIDE = 129;      // padded row stride of the staged tile
constexpr int LG_TILE = LG_IC * Q * LG_STRIDE;  // floats per staged Theta chunk
constexpr size_t LG_SMEM = 2 * (size_t)LG_TILE * sizeof(float) + 2 * (size_t)LG_BT * LG_IC;

__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

__global__ void __launch_bounds__(256)
k_logits_gather(const int8_t *__restrict__ msa, const float *__restrict__ theta,
                Dims d, float *__restrict__ L, const uint8_t *__restrict__ active)
{
    if (active) {  // skip row tiles whose sites need no evaluation
        bool any = false;
        const int rs0 = blockIdx.x * LG_ROWS;
        for (int r = rs0 / QP; r <= (rs0 + LG_ROWS - 1) / QP && r < d.N; ++r)
            any |= active[r] != 0;
        if (!any) return;
    }
    extern __shared__ float smem[];
    float *ths0 = smem;                                            // 2 x [IC*Q][129]
    int8_t *ss0 = (int8_t *)(smem + 2 * LG_TILE);                  // 2 x [BT][IC]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row0 = blockIdx.x * LG_ROWS;
    const int b0 = blockIdx.y * LG_BT;
    const int NQ = d.N * Q;

    // stage Theta[row0 .. +128][i0*Q .. +ncol] transposed (cp.async, 4 bytes
    // per element) and the chunk's states into buffer `buf`
    auto stage = [&](int buf, int i0) {
        float *ths = ths0 + buf * LG_TILE;
        int8_t *ss = ss0 + buf * LG_BT * LG_IC;
        const int ncol = min(LG_IC, d.N - i0) * Q;
        for (int e = tid; e < LG_ROWS * LG_IC * Q; e += blockDim.x) {
            const int cc = e % (LG_IC * Q);
            const int rr = e / (LG_IC * Q);
            float *dst = ths + cc * LG_STRIDE + rr;
            if (cc < ncol && row0 + rr < d.R)
                cp_async4(dst, theta + (size_t)(row0 + rr) * d.KP + i0 * Q + cc);
            else
                *dst = 0.0f;
        }
        for (int e = tid; e < LG_BT * LG_IC; e += blockDim.x) {
            const int ic = e % LG_IC, bb = e / LG_IC;
            const int b = b0 + bb, i = i0 + ic;
            ss[e] = (b < d.B && i < d.N) ? msa[(size_t)b * d.N + i] : 0;
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    float acc[LG_BPW][4];
#pragma unroll
    for (int u = 0; u < LG_BPW; ++u)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[u][j] = 0.0f;

    stage(0, 0);
    int buf = 0;
    for (int i0 = 0; i0 < d.N; i0 += LG_IC, buf ^= 1) {
        if (i0 + LG_IC < d.N) {
            stage(buf ^ 1, i0 + LG_IC);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const float *ths = ths0 + buf * LG_TILE;
        const int8_t *ssb = ss0 + buf * LG_BT * LG_IC;
        const int nic = min(LG_IC, d.N - i0);
        // positions outer, sequences inner: the 16 sequences' gathers of a
        // position are independent, so their loads are in flight together
        // (each accumulator still adds the positions in order)
        for (int ic = 0; ic < nic; ++ic) {
            int st[LG_BPW];
#pragma unroll
            for (int u = 0; u < LG_BPW; ++u) st[u] = ssb[(warp * LG_BPW + u) * LG_IC + ic];
#pragma unroll
            for (int u = 0; u < LG_BPW; ++u) {
                const float *col = ths + (ic * Q + st[u]) * LG_STRIDE + lane;
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[u][j] += col[32 * j];
            }
        }
        __syncthreads();  // the buffer is restaged two chunks on
    }
    // field column (its one-hot feature is 1 for every sequence)
    float hv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int row = row0 + lane + 32 * j;
        hv[j] = (row < d.R) ? theta[(size_t)row * d.KP + NQ] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < LG_BPW; ++u) {
        int b = b0 + warp * LG_BPW + u;
        if (b >= d.B) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int row = row0 + lane + 32 * j;
            if (row < d.R) L[(size_t)b * d.R + row] = acc[u][j] + hv[j];
        }
    }
}

constexpr int SM_WARPS = 8;

__global__ void __launch_bounds__(256)
k_softmax_resid(const int8_t *__restrict__ msa, const float *__restrict__ w,
                double beff, const float *__restrict__ L, Dims d,
                double *__restrict__ partial, float *__restrict__ D,
                const uint8_t *__restrict__ active)
{
    __shared__ double red[SM_WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.x * 32 + lane;
    const bool live = r < d.N && (!active || active[r]);
    const int nslices = gridDim.y * SM_WARPS;
    const int slice = blockIdx.y * SM_WARPS + warp;
    double obj = 0.0;
    if (live) {
        for (int b = slice; b < d.B; b += nslices) {
            const float *lr = L + (size_t)b * d.R + (size_t)r * QP;
            float l[Q];
            float mx = -INFINITY;
#pragma unroll
            for (int s = 0; s < Q; ++s) {
                l[s] = lr[s];
                mx = fmaxf(mx, l[s]);
            }
            float z = 0.0f;
#pragma unroll
            for (int s = 0; s < Q; ++s) z += expf(l[s] - mx);
            const float lse = mx + logf(z);
            const int sr = msa[(size_t)b * d.N + r];
            float lsr = l[0];
#pragma unroll
            for (int s = 1; s < Q; ++s)
                if (s == sr) lsr = l[s];
            const double wb = (double)w[b];
            obj += wb * (double)(lsr - lse);
            const float scale = (float)(wb / beff);
            float *dr = D + (size_t)b * d.R + (size_t)r * QP;
#pragma unroll
            for (int s = 0; s < Q; ++s)
                dr[s] = scale * (expf(l[s] - lse) - (s == sr ? 1.0f : 0.0f));
#pragma unroll
            for (int s = Q; s < QP; ++s) dr[s] = 0.0f;
        }
    }
    red[warp][lane] = obj;
    __syncthreads();
    if (warp == 0 && r < d.N) {
        double t = 0.0;
        for (int k = 0; k < SM_WARPS; ++k) t += red[k][lane];
        partial[(size_t)blockIdx.y * d.N + r] = t;
    }
}

__global__ void k_finish_objective(const double *__restrict__ partial,
                                   int slices, Dims d, double beff,
                                   const double *__restrict__ pen,
                                   double *__restrict__ f)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.N) return;
    double t = 0.0;
    for (int y = 0; y < slices; ++y) t += partial[(size_t)y * d.N + r];
    f[r] = -t / beff + (pen ? pen[r] : 0.0);
}

constexpr int GG_ROWS = 128;
constexpr int GG_IC = 8;     // positions per CTA (one per warp)
constexpr int GG_BT = 32;    // sequences per staged tile (two tiles in flight)

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N_PENDING>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N_PENDING) : "memory"); }

// Lane l of a warp owns rows row0 + 4l .. 4l + 3 (one float4 of a staged
// residual row); the residual tiles (32 sequences x 128 rows) are staged by
// cp.async into two buffers, so the next tile's loads overlap this one's sums.
__global__ void __launch_bounds__(256)
k_grad_gather(const int8_t *__restrict__ msa, const float *__restrict__ D,
              const float *__restrict__ theta, Dims d, double lambda_h,
              double lambda_Jp, float *__restrict__ G, const uint8_t *__restrict__ active)
{
    if (active) {
        bool any = false;
        const int rs0 = blockIdx.x * GG_ROWS;
        for (int r = rs0 / QP; r <= (rs0 + GG_ROWS - 1) / QP && r < d.N; ++r)
            any |= active[r] != 0;
        if (!any) return;
    }
    __shared__ __align__(16) float ds[2][GG_BT][GG_ROWS];
    __shared__ int8_t ss[2][GG_BT][GG_IC];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row0 = blockIdx.x * GG_ROWS;
    const int i0 = blockIdx.y * GG_IC;
    const int i = i0 + warp;
    const int NQ = d.N * Q;
    const bool field_warp = (blockIdx.y == 0 && warp == 0);

    // stage sequences b0 .. b0 + GG_BT - 1 into buffer `buf` (R is a multiple
    // of 4 and row0 of 128, so a float4 is either wholly inside or outside)
    auto stage = [&](int buf, int b0) {
        for (int e = tid; e < GG_BT * GG_ROWS / 4; e += blockDim.x) {
            const int bb = e / (GG_ROWS / 4), c4 = e % (GG_ROWS / 4);
            const int b = b0 + bb, row = row0 + 4 * c4;
            float *dst = &ds[buf][bb][4 * c4];
            if (b < d.B && row < d.R) cp_async16(dst, D + (size_t)b * d.R + row);
            else *(float4 *)dst = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int e = tid; e < GG_BT * GG_IC; e += blockDim.x) {
            const int ic = e % GG_IC, bb = e / GG_IC;
            const int b = b0 + bb, ii = i0 + ic;
            ss[buf][bb][ic] = (b < d.B && ii < d.N) ? msa[(size_t)b * d.N + ii] : 0;
        }
        cp_async_commit();
    };

    float acc[Q][4];
#pragma unroll
    for (int k = 0; k < Q; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[k][j] = 0.0f;
    float tot[4] = {0.0f, 0.0f, 0.0f, 0.0f};

    stage(0, 0);
    int buf = 0;
    for (int b0 = 0; b0 < d.B; b0 += GG_BT, buf ^= 1) {
        const bool more = b0 + GG_BT < d.B;
        if (more) {
            stage(buf ^ 1, b0 + GG_BT);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (i < d.N) {
            if (field_warp) {
#pragma unroll 4
                for (int bb = 0; bb < GG_BT; ++bb) {
                    const float4 v = *(const float4 *)&ds[buf][bb][4 * lane];
                    tot[0] += v.x;
                    tot[1] += v.y;
                    tot[2] += v.z;
                    tot[3] += v.w;
                }
            }
            // lane l holds the state of staged sequence l at this warp's
            // position; for each state the warp visits, in sequence order,
            // the sequences that show it (a uniform mask, no branch per
            // sequence) and adds their residual rows to that state's sums
            const int st = ss[buf][lane][warp];
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                unsigned mask = __ballot_sync(0xffffffffu, st == k);
                while (mask) {
                    const int bb = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const float4 v = *(const float4 *)&ds[buf][bb][4 * lane];
                    acc[k][0] += v.x;
                    acc[k][1] += v.y;
                    acc[k][2] += v.z;
                    acc[k][3] += v.w;
                }
            }
        }
        __syncthreads();  // the buffer is restaged two tiles on
    }
    // epilogue: add the penalty gradient 2 lambda theta; the diagonal block,
    // padding rows and padding columns are zero
    const float two_lj = (float)(2.0 * lambda_Jp), two_lh = (float)(2.0 * lambda_h);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int row = row0 + 4 * lane + j;
        if (row >= d.R) continue;
        const int r = row / QP, s = row % QP;
        const float *th = theta + (size_t)row * d.KP;
        float *g = G + (size_t)row * d.KP;
        if (i < d.N) {
            const bool zero = (s >= Q) || (i == r);
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const int c = i * Q + k;
                g[c] = zero ? 0.0f : acc[k][j] + two_lj * th[c];
            }
        }
        if (field_warp) g[NQ] = (s >= Q) ? 0.0f : tot[j] + two_lh * th[NQ];
        if (blockIdx.y == 0 && warp > 0)
            for (int c = NQ + warp; c < d.KP; c += 7) g[c] = 0.0f;
    }
}

}  // namespace

cudaError_t launch_logits_gather(const int8_t *msa, const float *theta,
                                 const Dims &d, float *L, const uint8_t *active,
                                 cudaStream_t st)
{
    static std::atomic<unsigned long long> attr{0};
    cudaError_t e = set_smem_limit_once((const void *)k_logits_gather, (int)LG_SMEM, attr);
    if (e) return e;
    dim3 grid((d.R + LG_ROWS - 1) / LG_ROWS, (d.B + LG_BT - 1) / LG_BT);
    k_logits_gather<<<grid, 256, LG_SMEM, st>>>(msa, theta, d, L, active);
    count_launches(1);
    return cudaGetLastError();
}

int softmax_slices(const Dims &d)
{
    // enough CTAs to fill the GPU, each warp looping over >= 16 sequences
    int ycap = (d.B + 16 * SM_WARPS - 1) / (16 * SM_WARPS);
    int xs = (d.N + 31) / 32;
    int y = (4 * num_sms() + xs - 1) / xs;
    if (y > ycap) y = ycap;
    if (y < 1) y = 1;
    return y;
}

cudaError_t launch_softmax_resid(const int8_t *msa, const float *w,
                                 double beff, const float *L, const Dims &d,
                                 double *partial, float *D, const uint8_t *active,
                                 cudaStream_t st)
{
    dim3 grid((d.N + 31) / 32, softmax_slices(d));
    k_softmax_resid<<<grid, 32 * SM_WARPS, 0, st>>>(msa, w, beff, L, d, partial, D, active);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_finish_objective(const double *partial, int slices,
                                    const Dims &d, double beff,
                                    const double *pen, double *f,
                                    cudaStream_t st)
{
    k_finish_objective<<<(d.N + 127) / 128, 128, 0, st>>>(partial, slices, d, beff, pen, f);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_grad_gather(const int8_t *msa, const float *D,
                               const float *theta, const Dims &d,
                               double lambda_h, double lambda_Jp, float *G,
                               const uint8_t *active, cudaStream_t st)
{
    dim3 grid((d.R + GG_ROWS - 1) / GG_ROWS, (d.N + GG_IC - 1) / GG_IC);
    k_grad_gather<<<grid, 256, 0, st>>>(msa, D, theta, d, lambda_h, lambda_Jp, G, active);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace plm
