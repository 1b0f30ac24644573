// k_tc.cu -- the split-BF16 tensor-core path (tcgen05 + TMA + TMEM, sm_103a).
//
// Logits (Eq. condpfinal for every site at once):
//     L[b][(r,s)] = sum_c X[b][c] Theta[(r,s)][c]
// with X the one-hot expansion of the MSA (exact in bf16) and Theta split as
// Theta_hi + Theta_lo, hi = RN_bf16(Theta), lo = RN_bf16(Theta - hi); both
// products accumulate into one FP32 accumulator in tensor memory.  The one-
// hot tile of X is written into shared memory by the CTA itself (never
// stored in HBM); the Theta tiles arrive by TMA.  The epilogue reads the
// accumulator row by row (one sequence per thread), does the log-softmax
// over the 21 states of each site, adds w_b (L[S_br] - lse) to a per-site
// FP64 partial of the objective (Eq. g_regdef2) and writes the residual
// D = (w_b / B_eff)(P - Y) (Eqs. g_gradh2, g_gradJ2) transposed and split
// into bf16 hi + lo.
//
// Gradient (Eq. g_gradJ2):  G[(r,s)][c] = sum_b D^T[(r,s)][b] X^T[c][b]
// with D^T hi/lo by TMA and the one-hot X^T tile built in shared memory from
// the transposed MSA; the epilogue adds 2 lambda Theta and zeroes the
// diagonal block and the padding.
//
// Both kernels: one 128-row output tile per CTA, 3-stage TMA/producer ->
// MMA pipeline on mbarriers, operands K-major with the 128-byte swizzle,
// M = 128, K = 16 per instruction.  Warp 0 issues TMA, warp 1 owns the
// tensor memory and issues the MMAs, warps 2-5 produce the one-hot operand
// and then run the epilogue.  Every mbarrier wait is bounded: on timeout
// the CTA records an error code, stops issuing, lets in-flight copies and
// MMAs finish, frees its tensor memory and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "plm_device.cuh"
#include "plm_internal.cuh"

namespace plm {

void *prof_start(void *ctx);
void prof_stop(void *ctx, const char *name, void *start);

namespace {

constexpr int TC_M = 128;
constexpr int TC_BK = 64;                  // K per stage: 64 bf16 = 128 bytes
constexpr int MAX_STAGES = 4;
constexpr int MAX_LG_SITES = 10;           // sites per logits tile: 2..10, even
constexpr int TMEM_COLS = 256;
constexpr int LG_A_BYTES = TC_M * TC_BK * 2;          // 16 KB
constexpr int GR_A_BYTES = TC_M * TC_BK * 2;          // 16 KB per 128 rows
constexpr int SMEM_BUDGET = 224 * 1024;  // pipeline bytes; + 1 KB alignment slack and the static
                                         // shared memory stay under the 227 KB per block
constexpr long long WAIT_CYCLES = 4000000000LL;        // ~2 s at 2 GHz

enum { ERR_TIMEOUT_TMA = 1 << 4, ERR_TIMEOUT_MMA = 1 << 5, ERR_TIMEOUT_PROD = 1 << 6,
       ERR_TIMEOUT_EPI = 1 << 7, ERR_TIMEOUT_SELFTEST = 1 << 8 };

// ---------------------------------------------------------------- PTX glue
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of the given parity.  Gives up (false) when
// the CTA's abort flag is raised or after WAIT_CYCLES, raising the flag and
// recording `code` in the global error word.
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                          int *err, int code)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > WAIT_CYCLES) {
            *abort_flag = 1;
            atomicOr(err, code);
            return false;
        }
    }
}

// wait without the abort short-cut (used to drain in-flight work)
__device__ bool mbar_drain(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > WAIT_CYCLES) return false;
    return true;
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// Shared-memory operand descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO); the leading offset is unused for this layout.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D f32, A and B bf16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v)
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

// sum over the warp of a float, carried as an unevaluated pair (hi, lo):
// each step adds the partner's pair with Knuth's two-sum, so the total keeps
// about 44 bits whatever the magnitudes
__device__ __forceinline__ double warp_sum_pair(float x)
{
    float hi = x, lo = 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float bh = __shfl_xor_sync(0xffffffffu, hi, o);
        const float bl = __shfl_xor_sync(0xffffffffu, lo, o);
        const float t = __fadd_rn(hi, bh);
        const float bp = __fsub_rn(t, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(bh, bp));
        hi = t;
        lo = __fadd_rn(__fadd_rn(lo, bl), e);
    }
    return (double)hi + (double)lo;
}

__device__ __forceinline__ void tmem_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void epi_bar256()
{
    asm volatile("bar.sync 1, 256;" ::: "memory");
}

__device__ __forceinline__ uint8_t *align1024(uint8_t *p)
{
    return (uint8_t *)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

// element (row, pos) of a K-major tile with 128-byte rows, 128B-swizzled
__device__ __forceinline__ uint32_t swz(int row, int chunk16)
{
    return (uint32_t)(row * 128 + ((chunk16 ^ (row & 7)) << 4));
}

// Kernel parameters of one batched launch: the family descriptors and one
// TMA map per family and operand (passed by value, read from param space).
struct LogitsParams {
    TcBatch b;
    int sites, ncols, stages, stage_bytes;  // tile: `sites` sites = ncols accumulator columns
    CUtensorMap hi[MAX_FAM], lo[MAX_FAM];
};

struct GradParams {
    TcBatch b;
    int rows, ncols, stages, stage_bytes;  // tile: rows (128 or 256) x ncols columns
    // k_tc_grad: 3-D maps (BP, 21 states, N sites), box (64, 21, GR_SITES);
    // k_tc_grad_pair: 2-D maps over the padded rows, box (64, 128)
    CUtensorMap dhi[MAX_FAM], dlo[MAX_FAM];
};

constexpr int GR_BOX_BYTES = TC_BK * 2 * Q * GR_SITES;  // one (64, 21, 6) box: 16128 bytes

// family owning global tile `tile` (tile0 ascending)
__device__ __forceinline__ int family_of(const TcBatch &b, int tile, bool grad)
{
    int f = 0;
    for (int k = 1; k < b.nfam; ++k)
        if ((grad ? b.f[k].tile0_grad : b.f[k].tile0_logits) <= tile) f = k;
    return f;
}

// the eight epilogue warps of the logits kernel
__device__ __forceinline__ void epi_bar_all()
{
    asm volatile("bar.sync 3, 256;" ::: "memory");
}

// tile t of the logits grid: family, sequence tile, site tile
__device__ __forceinline__ void lg_tile(const LogitsParams &P, int t, int &fi, int &tb, int &tr)
{
    fi = family_of(P.b, t, false);
    const FamDesc &F = P.b.f[fi];
    const int local = t - F.tile0_logits;
    const int nbt = F.BP / TC_M;
    tb = local % nbt;
    tr = local / nbt;
}

// does the tile hold a site that needs this evaluation?
__device__ __forceinline__ bool sites_active(const FamDesc &F, int r_lo, int r_hi)
{
    if (!F.active) return true;
    for (int r = r_lo; r <= r_hi && r < F.N; ++r)
        if (F.active[r]) return true;
    return false;
}

// ---------------------------------------------------------------- logits
// Persistent: one CTA per SM walks the tile list (stride gridDim.x).  Warp
// 0: TMA for Theta hi/lo; warp 1: TMEM (2 x 256 columns) and MMA issue;
// warps 2-5: one-hot producers; warps 6-13: epilogue, two groups of four
// warps (one per TMEM lane quarter) that take alternate sites of a tile.
// The accumulator is double-buffered, so a tile's epilogue overlaps the
// next tile's main loop.
constexpr int LG_THREADS = 448;
constexpr int LG_EPI = 256;  // epilogue threads
__global__ void __launch_bounds__(LG_THREADS, 1)
k_tc_logits(const __grid_constant__ LogitsParams P, int *__restrict__ err)
{
    extern __shared__ uint8_t dsmem[];
    uint8_t *smem = align1024(dsmem);
    const int LGS = P.sites, NST = P.stages, LGSTAGE = P.stage_bytes;
    const int LGB = P.ncols * TC_BK * 2;
    __shared__ __align__(8) uint64_t full_b[MAX_STAGES], full_a[MAX_STAGES], empty_[MAX_STAGES];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], mma_done;
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_sh;
    __shared__ double red[4][MAX_LG_SITES];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = P.b.ntiles_logits;

    if (threadIdx.x == 0) {
        for (int s = 0; s < MAX_STAGES; ++s) {
            mbar_init(&full_b[s], 1);
            mbar_init(&full_a[s], 4);  // one arrival per producer warp
            mbar_init(&empty_[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], LG_EPI);
        }
        mbar_init(&mma_done, 1);
        abort_sh = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(&tmem_sh, 2 * TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;

    if (warp == 0) {
        if (lane == 0) {
            long long kit = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                int fi, tb, tr;
                lg_tile(P, t, fi, tb, tr);
                const FamDesc &F = P.b.f[fi];
                if (!sites_active(F, tr * LGS, tr * LGS + LGS - 1)) continue;
                const int row0 = tr * LGS * QP, NK = F.KP / TC_BK;
                for (int kc = 0; kc < NK; ++kc, ++kit) {
                    const int s = (int)(kit % NST);
                    const long long n = kit / NST;
                    if (n > 0 &&
                        !mbar_wait(&empty_[s], (uint32_t)((n - 1) & 1), &abort_sh, err, ERR_TIMEOUT_TMA)) {
                        ok = false;
                        break;
                    }
                    uint8_t *st = smem + s * LGSTAGE;
                    mbar_expect_tx(&full_b[s], 2 * LGB);
                    tma_load_2d(st + LG_A_BYTES, &P.hi[fi], &full_b[s], kc * TC_BK, row0);
                    tma_load_2d(st + LG_A_BYTES + LGB, &P.lo[fi], &full_b[s], kc * TC_BK, row0);
                }
            }
            // let the copies still in flight land before the CTA can exit
            for (long long k = kit - NST < 0 ? 0 : kit - NST; k < kit; ++k)
                mbar_drain(&full_b[k % NST], (uint32_t)((k / NST) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(TC_M, P.ncols);
            long long kit = 0;
            int ti = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                int fi, tb, tr;
                lg_tile(P, t, fi, tb, tr);
                const FamDesc &F = P.b.f[fi];
                if (!sites_active(F, tr * LGS, tr * LGS + LGS - 1)) continue;
                const int a = ti & 1, use = ti >> 1;
                if (use > 0 &&
                    !mbar_wait(&acc_empty[a], (uint32_t)((use - 1) & 1), &abort_sh, err, ERR_TIMEOUT_MMA))
                    break;
                tc_fence_after();
                const uint32_t dt = tmem + a * TMEM_COLS;
                const int NK = F.KP / TC_BK;
                for (int kc = 0; kc < NK; ++kc, ++kit) {
                    const int s = (int)(kit % NST);
                    const uint32_t ph = (uint32_t)((kit / NST) & 1);
                    if (!mbar_wait(&full_b[s], ph, &abort_sh, err, ERR_TIMEOUT_MMA) ||
                        !mbar_wait(&full_a[s], ph, &abort_sh, err, ERR_TIMEOUT_MMA)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    uint8_t *st = smem + s * LGSTAGE;
                    const uint32_t aa = smem_u32(st);
                    const uint32_t bh = smem_u32(st + LG_A_BYTES);
                    const uint32_t bl = smem_u32(st + LG_A_BYTES + LGB);
#pragma unroll
                    for (int k = 0; k < TC_BK / 16; ++k)
                        mma_bf16(dt, sdesc(aa + 32 * k), sdesc(bh + 32 * k), idesc,
                                 (kc > 0 || k > 0) ? 1u : 0u);
#pragma unroll
                    for (int k = 0; k < TC_BK / 16; ++k)
                        mma_bf16(dt, sdesc(aa + 32 * k), sdesc(bl + 32 * k), idesc, 1u);
                    mma_commit(&empty_[s]);
                }
                if (!ok) break;
                mma_commit(&acc_full[a]);
                ++ti;
            }
            mma_commit(&mma_done);  // arrives when every MMA issued above has completed
        }
    } else if (warp < 6) {
        // ---- one-hot producers: thread p writes row p of X for each tile
        const int p = threadIdx.x - 64;
        long long kit = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            int fi, tb, tr;
            lg_tile(P, t, fi, tb, tr);
            const FamDesc &F = P.b.f[fi];
            if (!sites_active(F, tr * LGS, tr * LGS + LGS - 1)) continue;
            const int b = tb * TC_M + p;
            const bool valid = b < F.B;
            const int8_t *srow = F.msa + (size_t)(valid ? b : 0) * F.N;
            const int NK = F.KP / TC_BK, NQ = F.N * Q, N = F.N;
            // states of the (at most 5) positions a chunk of 64 columns
            // touches, fetched one chunk ahead
            auto fetch = [&](int kc, int (&st5)[5]) {
                const int i_lo = (kc * TC_BK) / Q;
#pragma unroll
                for (int u = 0; u < 5; ++u) {
                    const int i = i_lo + u;
                    st5[u] = (valid && i < N) ? (int)srow[i] : 0;
                }
            };
            int cur5[5], nxt5[5];
            fetch(0, cur5);
            for (int kc = 0; kc < NK; ++kc, ++kit) {
                const int s = (int)(kit % NST);
                const long long n = kit / NST;
                fetch(kc + 1 < NK ? kc + 1 : kc, nxt5);
                // the warp leaves together (it arrives once per stage)
                const bool got = n == 0 || mbar_wait(&empty_[s], (uint32_t)((n - 1) & 1), &abort_sh,
                                                     err, ERR_TIMEOUT_PROD);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                uint8_t *rowp = smem + s * LGSTAGE + p * 128;
                const uint4 z = make_uint4(0, 0, 0, 0);
                // rotate the chunk order by row so a warp's stores spread over the banks
#pragma unroll
                for (int j = 0; j < 8; ++j) *(uint4 *)(rowp + ((j + p) & 7) * 16) = z;
                if (valid) {
                    const int c0 = kc * TC_BK;
                    const int i_lo = c0 / Q;
#pragma unroll
                    for (int u = 0; u < 5; ++u) {
                        const int i = i_lo + u;
                        const int pos = i * Q + cur5[u] - c0;
                        if (i < N && pos >= 0 && pos < TC_BK)
                            *(uint16_t *)(rowp + ((((pos >> 3) ^ (p & 7)) << 4) | ((pos & 7) << 1))) =
                                0x3F80;
                    }
                    const int pf = NQ - c0;  // the field column: feature 1
                    if (pf >= 0 && pf < TC_BK)
                        *(uint16_t *)(rowp + ((((pf >> 3) ^ (p & 7)) << 4) | ((pf & 7) << 1))) =
                            0x3F80;
                }
                // every thread makes its stores visible to the tensor core's
                // proxy; then one arrival per warp
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(&full_a[s]);
#pragma unroll
                for (int u = 0; u < 5; ++u) cur5[u] = nxt5[u];
            }
        }
    } else {
        // ---- epilogue: one sequence per thread (its TMEM lane); group g
        // takes sites g, g + 2, ... of the tile.  Residual rows go straight
        // to global memory: for a fixed state row the 32 lanes of a warp
        // write 32 consecutive sequences (64 contiguous bytes).
        const int q4 = warp & 3;
        const int g = (warp - 6) >> 2;
        const int er = q4 * 32 + lane;
        int ti = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            int fi, tb, tr;
            lg_tile(P, t, fi, tb, tr);
            const FamDesc &F = P.b.f[fi];
            const int r0 = tr * LGS;
            if (!sites_active(F, r0, r0 + LGS - 1)) continue;
            const int a = ti & 1, use = ti >> 1;
            const int b0 = tb * TC_M, row0 = r0 * QP, BP = F.BP;
            const int eb = b0 + er;
            const bool ev = eb < F.B;
            // operands of the epilogue, fetched while the MMAs run
            const float wb = ev ? F.w[eb] : 0.0f;
            const float scale = (float)((double)wb * F.inv_beff);
            int sr[(MAX_LG_SITES + 1) / 2];
#pragma unroll
            for (int u = 0; u < (MAX_LG_SITES + 1) / 2; ++u) {
                const int r = r0 + g + 2 * u;
                sr[u] = (g + 2 * u < LGS && r < F.N) ? (int)F.msaT[(size_t)r * BP + eb] : -1;
            }
            const bool ok = mbar_wait(&acc_full[a], (uint32_t)(use & 1), &abort_sh, err, ERR_TIMEOUT_EPI);
            tc_fence_after();
            const uint32_t tl = tmem + a * TMEM_COLS + ((uint32_t)(q4 * 32) << 16);
            const int nmine = (LGS - g + 1) / 2;
            if (nmine == 0) {
                tc_fence_before();
                mbar_arrive(&acc_empty[a]);
            }
#pragma unroll
            for (int u = 0; u < (MAX_LG_SITES + 1) / 2; ++u) {
                if (u < nmine) {
                    const int j = g + 2 * u;
                    const int r = r0 + j;
                    const int srv = sr[u];
                    float l[24];
                    tmem_ld16(tl + j * QP, l);
                    tmem_ld8(tl + j * QP + 16, l + 16);
                    tmem_wait_ld();
                    if (u == nmine - 1) {
                        // this thread's last tensor-memory read of the tile
                        tc_fence_before();
                        mbar_arrive(&acc_empty[a]);
                    }
                    const bool live = ev && r < F.N && ok;
                    // numerically stable log-softmax over the q states (Eq. condpfinal)
                    float mx = l[0];
    #pragma unroll
                    for (int s2 = 1; s2 < Q; ++s2) mx = fmaxf(mx, l[s2]);
                    float z = 0.0f, lsr = 0.0f;
    #pragma unroll
                    for (int s2 = 0; s2 < Q; ++s2) {
                        if (s2 == srv) lsr = l[s2];
                        l[s2] = __expf(l[s2] - mx);
                        z += l[s2];
                    }
                    const float lse = mx + __logf(z);
                    const float iz = __fdividef(1.0f, z);
                    const double c = warp_sum_pair(live ? wb * (lsr - lse) : 0.0f);
                    if (lane == 0) red[q4][j] = c;
                    if (ok && r < F.N) {
                        __nv_bfloat16 *dh = F.dt_hi + (size_t)(row0 + j * QP) * BP + eb;
                        __nv_bfloat16 *dl = F.dt_lo + (size_t)(row0 + j * QP) * BP + eb;
    #pragma unroll
                        for (int s2 = 0; s2 < QP; ++s2) {
                            float dv = 0.0f;
                            if (s2 < Q && ev)
                                dv = scale * (l[s2] * iz - (s2 == srv ? 1.0f : 0.0f));
                            const __nv_bfloat16 hi = __float2bfloat16_rn(dv);
                            dh[(size_t)s2 * BP] = hi;
                            dl[(size_t)s2 * BP] = __float2bfloat16_rn(dv - __bfloat162float(hi));
                        }
                    }
                }
            }
            epi_bar_all();
            const int t256 = threadIdx.x - 192;
            if (t256 < LGS && r0 + t256 < F.N && ok)
                F.partial[(size_t)tb * F.N + r0 + t256] =
                    ((red[0][t256] + red[1][t256]) + red[2][t256]) + red[3][t256];
            epi_bar_all();
            ++ti;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        // every MMA must be complete before the tensor memory is released
        if (lane == 0) mbar_drain(&mma_done, 0);
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, 2 * TMEM_COLS);
    }
}

// ---------------------------------------------------------------- CTA pair
// The logits on a pair of CTAs (a 2-CTA cluster, tcgen05 cta_group::2):
// one MMA instruction computes a 256-sequence x NMMA-column product, each
// CTA holding its own 128 sequences' one-hot rows (A) and half of the Theta
// rows (B), each accumulating its 128 rows in its own tensor memory.  Half
// the Theta bytes per SM let a pipeline stage carry 128 of K (16 MMAs per
// stage handshake instead of 8).  Sites are packed 21 columns apart (no
// padding rows): a CTA's B half holds SH sites (21 SH rows, the rest of the
// NMMA/2 rows unused), loaded by one 3-D TMA box per operand and K atom.
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// the shared::cluster address of `p` (this CTA's shared memory) in CTA `rank`
__device__ __forceinline__ uint32_t cluster_addr(const void *p, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t caddr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr)
                 : "memory");
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// 3-D box into this CTA's shared memory, completion counted on the barrier
// at cluster address `bar_cl` (the leader CTA's)
__device__ __forceinline__ void tma_load_3d_pair(void *dst, const CUtensorMap *map, uint32_t bar_cl,
                                                 int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar_cl)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc_pair(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish_pair()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void mma_bf16_pair(uint32_t d_tmem, uint64_t a, uint64_t b,
                                              uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrives (when the MMAs issued so far are complete) on the barrier at the
// same shared-memory offset in both CTAs of the pair
__device__ __forceinline__ void mma_commit_pair(uint64_t *bar)
{
    const uint16_t mask = 3;
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
        "[%0], %1;" ::"r"(smem_u32(bar)),
        "h"(mask)
        : "memory");
}

struct PairParams {
    TcBatch b;
    int stages, stage_bytes;   // a stage holds one or two K atoms of 64
    CUtensorMap hi[MAX_FAM], lo[MAX_FAM];  // 3-D maps (KP, 21 states, N sites), box (64, 21, SH)
};

constexpr int LP_THREADS = 448;

template <int SH, int ATOMS>
struct PairShape {
    static constexpr int SITES = 2 * SH;                        // sites per tile
    static constexpr int NMMA = (SITES * Q + 15) / 16 * 16;     // MMA N (accumulator columns)
    static constexpr int NH = NMMA / 2;                         // B rows per CTA
    static constexpr int A_ATOM = TC_M * TC_BK * 2;             // 16 KB
    static constexpr int B_ATOM = (NH * TC_BK * 2 + 1023) / 1024 * 1024;
    static constexpr int STAGE = ATOMS * (A_ATOM + 2 * B_ATOM);  // ATOMS K atoms of 64
    static constexpr int BOX_BYTES = TC_BK * 2 * Q * SH;        // one (64, 21, SH) box
};

// tile t of the pair grid: family, 256-sequence tile, site group
__device__ __forceinline__ void lp_tile(const TcBatch &b, int t, int sites, int &fi, int &ptb,
                                        int &tr)
{
    fi = family_of(b, t, false);
    const FamDesc &F = b.f[fi];
    const int local = t - F.tile0_logits;
    const int nbt2 = (F.BP / TC_M + 1) / 2;
    ptb = local % nbt2;
    tr = local / nbt2;
}

// Roles (both CTAs): warp 0 TMA of this CTA's Theta half, signalled on the
// leader's barrier; warp 1 tensor memory (both) and MMA issue (leader
// only); warps 2-5 one-hot producers of this CTA's 128 sequences, arriving
// on the leader's barrier; warps 6-13 epilogue of this CTA's accumulator
// rows, two groups of four warps taking the two site halves.
template <int SH, int LP_ATOMS>
__global__ void __launch_bounds__(LP_THREADS, 1)
k_tc_logits_pair(const __grid_constant__ PairParams P, int *__restrict__ err)
{
    using S = PairShape<SH, LP_ATOMS>;
    extern __shared__ uint8_t dsmem[];
    uint8_t *smem = align1024(dsmem);
    const int NST = P.stages;
    __shared__ __align__(8) uint64_t full_[MAX_STAGES], empty_[MAX_STAGES];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], mma_done;
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_sh;
    __shared__ double red[4][S::SITES];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
    const int ntiles = P.b.ntiles_logits;

    if (threadIdx.x == 0) {
        for (int s = 0; s < MAX_STAGES; ++s) {
            mbar_init(&full_[s], 1 + 2 * 4);  // leader's TMA arrival + 4 producer warps per CTA
            mbar_init(&empty_[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], 2 * 8);  // 8 epilogue warps per CTA
        }
        mbar_init(&mma_done, 1);
        abort_sh = 0;
        fence_mbar_init();
    }
    __syncthreads();
    cluster_sync_all();  // both CTAs' barriers exist before any remote arrival
    if (warp == 1) {
        // one warp of each CTA allocates, together, the same columns in both
        tmem_alloc_pair(&tmem_sh, 2 * TMEM_COLS);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;

    if (warp == 0) {
        if (lane == 0) {
            long long kit = 0;
            bool ok = true;
            for (int t = pair; t < ntiles && ok; t += npairs) {
                int fi, ptb, tr;
                lp_tile(P.b, t, S::SITES, fi, ptb, tr);
                const FamDesc &F = P.b.f[fi];
                if (!sites_active(F, tr * S::SITES, tr * S::SITES + S::SITES - 1)) continue;
                const int site0 = tr * S::SITES + (int)rank * SH;
                const int NA = F.KP / TC_BK;
                for (int ka = 0; ka < NA; ka += LP_ATOMS, ++kit) {
                    const int na = NA - ka < LP_ATOMS ? NA - ka : LP_ATOMS;
                    const int s = (int)(kit % NST);
                    const long long n = kit / NST;
                    if (n > 0 &&
                        !mbar_wait(&empty_[s], (uint32_t)((n - 1) & 1), &abort_sh, err, ERR_TIMEOUT_TMA)) {
                        ok = false;
                        break;
                    }
                    uint8_t *st = smem + s * S::STAGE;
                    const uint32_t bar = cluster_addr(&full_[s], 0);
                    if (leader) mbar_expect_tx(&full_[s], 2 * na * 2 * S::BOX_BYTES);
                    for (int a = 0; a < na; ++a) {
                        uint8_t *bh = st + LP_ATOMS * S::A_ATOM + 2 * a * S::B_ATOM;
                        tma_load_3d_pair(bh, &P.hi[fi], bar, (ka + a) * TC_BK, 0, site0);
                        tma_load_3d_pair(bh + S::B_ATOM, &P.lo[fi], bar, (ka + a) * TC_BK, 0, site0);
                    }
                }
            }
            // the leader's barriers count both CTAs' copies: let the copies
            // still in flight land before either CTA can exit
            if (leader)
                for (long long k = kit - NST < 0 ? 0 : kit - NST; k < kit; ++k)
                    mbar_drain(&full_[k % NST], (uint32_t)((k / NST) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            const uint32_t idesc = idesc_bf16(2 * TC_M, S::NMMA);
            long long kit = 0;
            int ti = 0;
            bool ok = true;
            for (int t = pair; t < ntiles && ok; t += npairs) {
                int fi, ptb, tr;
                lp_tile(P.b, t, S::SITES, fi, ptb, tr);
                const FamDesc &F = P.b.f[fi];
                if (!sites_active(F, tr * S::SITES, tr * S::SITES + S::SITES - 1)) continue;
                const int a = ti & 1, use = ti >> 1;
                if (use > 0 && !mbar_wait(&acc_empty[a], (uint32_t)((use - 1) & 1), &abort_sh,
                                                  err, ERR_TIMEOUT_MMA))
                    break;
                tc_fence_after();
                const uint32_t dt = tmem + a * TMEM_COLS;
                const int NA = F.KP / TC_BK;
                for (int ka = 0; ka < NA; ka += LP_ATOMS, ++kit) {
                    const int na = NA - ka < LP_ATOMS ? NA - ka : LP_ATOMS;
                    const int s = (int)(kit % NST);
                    const uint32_t ph = (uint32_t)((kit / NST) & 1);
                    if (!mbar_wait(&full_[s], ph, &abort_sh, err, ERR_TIMEOUT_MMA)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    uint8_t *st = smem + s * S::STAGE;
                    for (int a2 = 0; a2 < na; ++a2) {
                        const uint32_t aa = smem_u32(st + a2 * S::A_ATOM);
                        const uint32_t bh = smem_u32(st + LP_ATOMS * S::A_ATOM + 2 * a2 * S::B_ATOM);
                        const uint32_t bl = bh + S::B_ATOM;
#pragma unroll
                        for (int k = 0; k < TC_BK / 16; ++k)
                            mma_bf16_pair(dt, sdesc(aa + 32 * k), sdesc(bh + 32 * k), idesc,
                                          (ka > 0 || a2 > 0 || k > 0) ? 1u : 0u);
#pragma unroll
                        for (int k = 0; k < TC_BK / 16; ++k)
                            mma_bf16_pair(dt, sdesc(aa + 32 * k), sdesc(bl + 32 * k), idesc, 1u);
                    }
                    mma_commit_pair(&empty_[s]);
                }
                if (!ok) break;
                mma_commit_pair(&acc_full[a]);
                ++ti;
            }
            mma_commit_pair(&mma_done);  // arrives in both CTAs when every MMA above is complete
        }
    } else if (warp < 6) {
        // ---- one-hot producers: thread p writes row p of X (this CTA's
        // 128 sequences) for each K atom of a stage
        const int p = threadIdx.x - 64;
        long long kit = 0;
        bool ok = true;
        for (int t = pair; t < ntiles && ok; t += npairs) {
            int fi, ptb, tr;
            lp_tile(P.b, t, S::SITES, fi, ptb, tr);
            const FamDesc &F = P.b.f[fi];
            if (!sites_active(F, tr * S::SITES, tr * S::SITES + S::SITES - 1)) continue;
            const int b = (2 * ptb + (int)rank) * TC_M + p;
            const bool valid = b < F.B;
            const int8_t *srow = F.msa + (size_t)(valid ? b : 0) * F.N;
            const int NA = F.KP / TC_BK, NQ = F.N * Q, N = F.N;
            for (int ka = 0; ka < NA; ka += LP_ATOMS, ++kit) {
                const int na = NA - ka < LP_ATOMS ? NA - ka : LP_ATOMS;
                const int s = (int)(kit % NST);
                const long long n = kit / NST;
                // states of the (at most 8) positions the stage's columns touch,
                // read before the wait so the loads overlap it
                const int i_lo = (ka * TC_BK) / Q;
                int st8[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i_lo + u;
                    st8[u] = (valid && i < N) ? (int)srow[i] : 0;
                }
                const bool got = n == 0 || mbar_wait(&empty_[s], (uint32_t)((n - 1) & 1), &abort_sh,
                                                     err, ERR_TIMEOUT_PROD);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                for (int a = 0; a < na; ++a) {
                    uint8_t *rowp = smem + s * S::STAGE + a * S::A_ATOM + p * 128;
                    const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll
                    for (int j = 0; j < 8; ++j) *(uint4 *)(rowp + ((j + p) & 7) * 16) = z;
                    if (valid) {
                        const int c0 = (ka + a) * TC_BK;
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int i = i_lo + u;
                            const int pos = i * Q + st8[u] - c0;
                            if (i < N && pos >= 0 && pos < TC_BK)
                                *(uint16_t *)(rowp + ((((pos >> 3) ^ (p & 7)) << 4) | ((pos & 7) << 1))) =
                                    0x3F80;
                        }
                        const int pf = NQ - c0;  // the field column: feature 1
                        if (pf >= 0 && pf < TC_BK)
                            *(uint16_t *)(rowp + ((((pf >> 3) ^ (p & 7)) << 4) | ((pf & 7) << 1))) =
                                0x3F80;
                    }
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(cluster_addr(&full_[s], 0));
            }
        }
    } else {
        // ---- epilogue: one sequence per thread (its tensor-memory lane);
        // group g takes the sites of B half g (columns g NH + 21 j)
        const int q4 = warp & 3;
        const int g = (warp - 6) >> 2;
        const int er = q4 * 32 + lane;
        int ti = 0;
        for (int t = pair; t < ntiles; t += npairs) {
            int fi, ptb, tr;
            lp_tile(P.b, t, S::SITES, fi, ptb, tr);
            const FamDesc &F = P.b.f[fi];
            const int r0 = tr * S::SITES;
            if (!sites_active(F, r0, r0 + S::SITES - 1)) continue;
            const int a = ti & 1, use = ti >> 1;
            const int tb = 2 * ptb + (int)rank;    // this CTA's 128-sequence tile
            const bool tile_ok = tb < F.BP / TC_M;  // the last pair may have one tile
            const int BP = F.BP;
            const int eb = tb * TC_M + er;
            const bool ev = tile_ok && eb < F.B;
            const float wb = ev ? F.w[eb] : 0.0f;
            const float scale = (float)((double)wb * F.inv_beff);
            int sr[SH];
#pragma unroll
            for (int j = 0; j < SH; ++j) {
                const int r = r0 + g * SH + j;
                sr[j] = (tile_ok && r < F.N) ? (int)F.msaT[(size_t)r * BP + eb] : -1;
            }
            const bool ok = mbar_wait(&acc_full[a], (uint32_t)(use & 1), &abort_sh, err, ERR_TIMEOUT_EPI);
            tc_fence_after();
            const uint32_t tl = tmem + a * TMEM_COLS + ((uint32_t)(q4 * 32) << 16);
#pragma unroll
            for (int j = 0; j < SH; ++j) {
                const int jj = g * SH + j;         // site within the tile
                const int r = r0 + jj;
                const int cl = 21 * j;             // column within the half
                const int ws = cl & ~7, o = cl & 7;
                float l[32];
                tmem_ld16(tl + g * S::NH + ws, l);
                if (o + Q > 24) tmem_ld16(tl + g * S::NH + ws + 16, l + 16);
                else tmem_ld8(tl + g * S::NH + ws + 16, l + 16);
                tmem_wait_ld();
                if (j == SH - 1) {
                    // this warp's last tensor-memory read of the tile
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive_cluster(cluster_addr(&acc_empty[a], 0));
                }
                const int srv = sr[j];
                const bool live = ev && r < F.N && ok;
                float mx = l[o];
#pragma unroll
                for (int s2 = 1; s2 < Q; ++s2) mx = fmaxf(mx, l[o + s2]);
                float z = 0.0f, lsr = 0.0f;
#pragma unroll
                for (int s2 = 0; s2 < Q; ++s2) {
                    if (s2 == srv) lsr = l[o + s2];
                    l[o + s2] = __expf(l[o + s2] - mx);
                    z += l[o + s2];
                }
                const float lse = mx + __logf(z);
                const float iz = __fdividef(1.0f, z);
                const double c = warp_sum_pair(live ? wb * (lsr - lse) : 0.0f);
                if (lane == 0) red[q4][jj] = c;
                if (ok && tile_ok && r < F.N) {
                    // the residual's rows of this site (the QP - Q padding rows
                    // only feed gradient rows that the gradient kernel zeroes,
                    // so they are not written)
                    __nv_bfloat16 *dh = F.dt_hi + (size_t)(r * QP) * BP + eb;
                    __nv_bfloat16 *dl = F.dt_lo + (size_t)(r * QP) * BP + eb;
#pragma unroll
                    for (int s2 = 0; s2 < Q; ++s2) {
                        float dv = 0.0f;
                        if (ev) dv = scale * (l[o + s2] * iz - (s2 == srv ? 1.0f : 0.0f));
                        const __nv_bfloat16 hi = __float2bfloat16_rn(dv);
                        dh[(size_t)s2 * BP] = hi;
                        dl[(size_t)s2 * BP] = __float2bfloat16_rn(dv - __bfloat162float(hi));
                    }
                }
            }
            epi_bar_all();
            const int t256 = threadIdx.x - 192;
            if (t256 < S::SITES && r0 + t256 < F.N && ok && tile_ok)
                F.partial[(size_t)tb * F.N + r0 + t256] =
                    ((red[0][t256] + red[1][t256]) + red[2][t256]) + red[3][t256];
            epi_bar_all();
            ++ti;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1 && lane == 0) mbar_drain(&mma_done, 0);  // every MMA into this CTA's memory
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();  // no arrival or copy of either CTA is still in flight
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, 2 * TMEM_COLS);
    }
    cluster_sync_all();
}

// ---------------------------------------------------------------- gradient
// One rows x ncols tile per CTA (measured faster here than a persistent
// variant: with ~1.5 tiles per SM there is little epilogue to overlap, and
// the whole-tile shared-memory staging of the epilogue writes G coalesced).
// The rows are packed by site: each 128-row accumulator holds GR_SITES
// sites x 21 states (rows 126 and 127 unused), loaded by one 3-D box per
// operand that skips the padding rows of the residual, so no MMA is spent
// on them; the epilogue writes the padding rows of G as zeros.
// Warp 0: TMA for D^T hi/lo; warp 1: TMEM and MMA issue; warps 2-9: the
// one-hot X^T producers (one operand row per thread: with one warp per
// scheduler the producers were latency bound), then the epilogue.
constexpr int GR_THREADS = 320;
constexpr int GR_PROD = 256;
__global__ void __launch_bounds__(GR_THREADS, 1)
k_tc_grad(const __grid_constant__ GradParams P, float two_lh, float two_lj, int *__restrict__ err)
{
    const int fi = family_of(P.b, blockIdx.x, true);
    const FamDesc &F = P.b.f[fi];
    const CUtensorMap &tm_dhi = P.dhi[fi];
    const CUtensorMap &tm_dlo = P.dlo[fi];
    const int8_t *__restrict__ msaT = F.msaT;
    const float *__restrict__ theta = F.theta;
    float *__restrict__ G = F.G;
    const int BP = F.BP;
    Dims d;
    d.B = F.B;
    d.N = F.N;
    d.KP = F.KP;
    d.R = F.R;
    d.K = F.N * Q + 1;
    const int local = blockIdx.x - F.tile0_grad;
    const int GRN = P.ncols, NST = P.stages, GRSTAGE = P.stage_bytes;
    // MR rows = MH halves of 128; half h accumulates in tensor-memory
    // columns [256 h, 256 h + GRN) from the A rows at h * GR_A_BYTES
    const int MR = P.rows, MH = MR / TC_M, ABYTES = MH * GR_A_BYTES;
    const int nct = (d.KP + GRN - 1) / GRN;
    extern __shared__ uint8_t dsmem[];
    uint8_t *smem = align1024(dsmem);
    __shared__ __align__(8) uint64_t full_b[MAX_STAGES], full_a[MAX_STAGES], empty_[MAX_STAGES], acc_full;
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = (local % nct) * GRN;
    const int sg0 = (local / nct) * MH * GR_SITES;  // first site of the tile
    if (F.active) {
        bool any = false;
        for (int r = sg0; r < sg0 + MH * GR_SITES && r < F.N; ++r)
            any |= F.active[r] != 0;
        if (!any) return;
    }
    const int NK = BP / TC_BK;
    const int NQ = d.N * Q;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full_b[s], 1);
            mbar_init(&full_a[s], GR_PROD / 32);  // one arrival per producer warp
            mbar_init(&empty_[s], 1);
        }
        mbar_init(&acc_full, 1);
        abort_sh = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(&tmem_sh, MH * TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kc = 0; kc < NK; ++kc) {
                const int s = kc % NST, n = kc / NST;
                if (n > 0 && !mbar_wait(&empty_[s], (n - 1) & 1, &abort_sh, err, ERR_TIMEOUT_TMA))
                    break;
                uint8_t *st = smem + s * GRSTAGE;
                // sites beyond N read as zeros; the full box is counted
                mbar_expect_tx(&full_b[s], 2 * MH * GR_BOX_BYTES);
                for (int h = 0; h < MH; ++h) {
                    tma_load_3d(st + h * GR_A_BYTES, &tm_dhi, &full_b[s], kc * TC_BK, 0,
                                sg0 + h * GR_SITES);
                    tma_load_3d(st + ABYTES + h * GR_A_BYTES, &tm_dlo, &full_b[s], kc * TC_BK,
                                0, sg0 + h * GR_SITES);
                }
                issued = kc + 1;
            }
            for (int kc = issued - NST < 0 ? 0 : issued - NST; kc < issued; ++kc)
                mbar_drain(&full_b[kc % NST], (kc / NST) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(TC_M, GRN);
            for (int kc = 0; kc < NK; ++kc) {
                const int s = kc % NST, n = kc / NST;
                if (!mbar_wait(&full_b[s], n & 1, &abort_sh, err, ERR_TIMEOUT_MMA)) break;
                if (!mbar_wait(&full_a[s], n & 1, &abort_sh, err, ERR_TIMEOUT_MMA)) break;
                tc_fence_after();
                uint8_t *st = smem + s * GRSTAGE;
                const uint32_t bx = smem_u32(st + 2 * ABYTES);
                for (int h = 0; h < MH; ++h) {
                    const uint32_t ah = smem_u32(st + h * GR_A_BYTES);
                    const uint32_t al = smem_u32(st + ABYTES + h * GR_A_BYTES);
                    const uint32_t dt = tmem + h * TMEM_COLS;
#pragma unroll
                    for (int k = 0; k < TC_BK / 16; ++k)
                        mma_bf16(dt, sdesc(ah + 32 * k), sdesc(bx + 32 * k), idesc,
                                 (kc > 0 || k > 0) ? 1u : 0u);
#pragma unroll
                    for (int k = 0; k < TC_BK / 16; ++k)
                        mma_bf16(dt, sdesc(al + 32 * k), sdesc(bx + 32 * k), idesc, 1u);
                }
                mma_commit(&empty_[s]);
            }
            mma_commit(&acc_full);
        }
    } else {
        // ---- one-hot X^T producer: thread p writes operand row p
        const int p = threadIdx.x - 64;
        const int c = c0 + p;
        int src_i = 0;
        uint32_t kk = 0xFFu;  // never equals a stored state (0..20, or 0x7F padding)
        if (c < NQ) {
            src_i = c / Q;
            kk = (uint32_t)(c % Q);
        } else if (c == NQ) {
            src_i = d.N;  // the all-ones row of msaT
            kk = 0;
        }
        kk *= 0x01010101u;
        const bool prow = p < GRN;
        // the next stage's MSA bytes are fetched while the current stage is
        // written, so the global-load latency overlaps the pipeline
        const uint4 *srcT = (const uint4 *)(msaT + (size_t)src_i * BP);
        uint4 cur[4], nxt[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) cur[q] = __ldg(srcT + q);
        for (int kc = 0; kc < NK; ++kc) {
            const int s = kc % NST, n = kc / NST;
            const int kn = kc + 1 < NK ? kc + 1 : kc;
#pragma unroll
            for (int q = 0; q < 4; ++q) nxt[q] = __ldg(srcT + (size_t)kn * (TC_BK / 16) + q);
            // the warp leaves together (it arrives once per stage)
            const bool got = n == 0 || mbar_wait(&empty_[s], (n - 1) & 1, &abort_sh, err,
                                                 ERR_TIMEOUT_PROD);
            if (!__all_sync(0xffffffffu, got)) break;
            uint8_t *bt = smem + s * GRSTAGE + 2 * ABYTES;
            if (prow) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {  // 16 sequences per word group
                    const uint4 x = cur[q];
                    const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
                    uint32_t o[8];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const uint32_t m = __vcmpeq4(xs[t], kk);
                        o[2 * t] = __byte_perm(m, 0, 0x1100) & 0x3F803F80u;
                        o[2 * t + 1] = __byte_perm(m, 0, 0x3322) & 0x3F803F80u;
                    }
                    *(uint4 *)(bt + swz(p, 2 * q)) = make_uint4(o[0], o[1], o[2], o[3]);
                    *(uint4 *)(bt + swz(p, 2 * q + 1)) = make_uint4(o[4], o[5], o[6], o[7]);
                }
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full_a[s]);
#pragma unroll
            for (int q = 0; q < 4; ++q) cur[q] = nxt[q];
        }

        // ---- epilogue: TMEM -> shared (rows padded to 260 floats so the
        // lane-per-row stores spread over the banks), then a coalesced pass
        // adds 2 lambda Theta, applies the masks and writes G.
        const int q4 = warp & 3;
        const int half = (warp - 2) >> 2;  // column half of the tile
        const int trow = q4 * 32 + lane;
        const bool ok = mbar_wait(&acc_full, 0, &abort_sh, err, ERR_TIMEOUT_EPI);
        tc_fence_after();
        const int GS = GRN + 4;
        float *acc_s = (float *)smem;  // [128][GS]
        const int NG = GRN / 16, ng0 = (NG + 1) / 2;  // 16-column groups; half 0 takes ng0
        for (int h = 0; h < MH; ++h) {
        const uint32_t tl = tmem + h * TMEM_COLS + ((uint32_t)(q4 * 32) << 16);
        const int sh0 = sg0 + h * GR_SITES;  // first site of this half
#pragma unroll 1
        for (int cc = half ? ng0 : 0; cc < (half ? NG : ng0); ++cc) {
            float v[16];
            tmem_ld16(tl + cc * 16, v);
            tmem_wait_ld();
            float4 *dst = (float4 *)(acc_s + trow * GS + cc * 16);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
        epi_bar256();
        const int t = threadIdx.x - 64;
        constexpr int UNR = 4;
        // accumulator row rr of this half: site sh0 + rr / Q, state rr % Q
        constexpr int HR = GR_SITES * Q;  // 126 rows in use
        for (int e0 = t; e0 < HR * (GRN / 4); e0 += GR_PROD * UNR) {
            float4 th[UNR];
            bool live[UNR];
            int rowk[UNR];
#pragma unroll
            for (int k = 0; k < UNR; ++k) {  // issue all loads first
                const int e = e0 + GR_PROD * k;
                const int rr = e / (GRN / 4), c4 = e % (GRN / 4);
                const int r = sh0 + rr / Q, cb = c0 + 4 * c4;
                rowk[k] = r * QP + rr % Q;
                live[k] = ok && e < HR * (GRN / 4) && r < d.N && cb < d.KP;
                th[k] = live[k] ? *(const float4 *)(theta + (size_t)rowk[k] * d.KP + cb)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int k = 0; k < UNR; ++k) {
                if (!live[k]) continue;
                const int e = e0 + GR_PROD * k;
                const int rr = e / (GRN / 4), c4 = e % (GRN / 4);
                const int r = sh0 + rr / Q, cb = c0 + 4 * c4;
                const float4 a = *(const float4 *)(acc_s + rr * GS + 4 * c4);
                const float av[4] = {a.x, a.y, a.z, a.w};
                const float tv[4] = {th[k].x, th[k].y, th[k].z, th[k].w};
                float o[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c = cb + u;
                    float val;
                    if (c > NQ || (c >= r * Q && c < r * Q + Q)) val = 0.0f;
                    else if (c == NQ) val = av[u] + two_lh * tv[u];
                    else val = av[u] + two_lj * tv[u];
                    o[u] = val;
                }
                *(float4 *)(G + (size_t)rowk[k] * d.KP + cb) = make_float4(o[0], o[1], o[2], o[3]);
            }
        }
        // the padding rows (states Q..QP-1) of this half's sites
        constexpr int PR = GR_SITES * (QP - Q);
        for (int e = t; e < PR * (GRN / 4); e += GR_PROD) {
            const int pr = e / (GRN / 4), c4 = e % (GRN / 4);
            const int r = sh0 + pr / (QP - Q), cb = c0 + 4 * c4;
            if (ok && r < d.N && cb < d.KP)
                *(float4 *)(G + (size_t)(r * QP + Q + pr % (QP - Q)) * d.KP + cb) =
                    make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (h + 1 < MH) epi_bar256();  // the staging buffer is reused by the next half
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        // every MMA must be complete before the tensor memory is released
        if (lane == 0) mbar_drain(&acc_full, 0);
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, MH * TMEM_COLS);
    }
}

// ---------------------------------------------------------------- gradient, CTA pair
// The gradient on 2-CTA clusters, persistent: a pair tile is 256 rows (128
// per CTA, each CTA's own D^T rows by TMA into its own accumulator) x ncols
// columns, each CTA building the one-hot X^T rows of half of the columns.
// A stage holds 128 of K (two 64-wide atoms).  Roles: warp 0 TMA (both
// CTAs, counted on the leader's barrier), warp 1 tensor memory (both) and
// MMA issue (leader), warps 2-9 one-hot producers (thread p: column p % 128
// of this CTA's half, K atom p / 128 of each stage), warps 10-13 the
// epilogue of this CTA's 128 rows (one row per thread: 2 lambda Theta added,
// masks applied, G written from registers).  Two accumulators, so a tile's
// epilogue overlaps the next tile's MMAs.
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, uint32_t bar_cl,
                                                 int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar_cl)
        : "memory");
}

constexpr int GP_ATOMS = 2;  // K atoms of 64 per stage
constexpr int GP_THREADS = 448;

// pair tile t: family, first row (of the 256), first column
__device__ __forceinline__ void gp_tile(const GradParams &P, int t, int &fi, int &rs0, int &c0)
{
    fi = family_of(P.b, t, true);
    const FamDesc &F = P.b.f[fi];
    const int local = t - F.tile0_grad;
    const int nct = (F.KP + P.ncols - 1) / P.ncols;
    c0 = (local % nct) * P.ncols;
    rs0 = (local / nct) * 2 * TC_M;
}

__device__ __forceinline__ bool rows_active(const FamDesc &F, int rs0)
{
    if (!F.active) return true;
    for (int r = rs0 / QP; r <= (rs0 + 2 * TC_M - 1) / QP && r < F.N; ++r)
        if (F.active[r]) return true;
    return false;
}

__global__ void __launch_bounds__(GP_THREADS, 1)
k_tc_grad_pair(const __grid_constant__ GradParams P, float two_lh, float two_lj, int *__restrict__ err)
{
    const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int ntiles = P.b.ntiles_grad;
    const int GRN = P.ncols, NST = P.stages, GRSTAGE = P.stage_bytes;
    const int HN = GRN / 2;                   // one-hot columns built by this CTA
    const int A_BYTES = GR_A_BYTES;           // 128 rows x 64 of K, bf16
    const int B_BYTES = HN * TC_BK * 2;
    const int B_OFF = GP_ATOMS * 2 * A_BYTES;  // stage: A_hi a0 | A_lo a0 | A_hi a1 | A_lo a1 | B a0 | B a1
    extern __shared__ uint8_t dsmem[];
    uint8_t *smem = align1024(dsmem);
    __shared__ __align__(8) uint64_t full_[MAX_STAGES], empty_[MAX_STAGES];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], mma_done;
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_sh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < MAX_STAGES; ++s) {
            mbar_init(&full_[s], 1 + 2 * (GR_PROD / 32));  // leader's TMA + 8 producer warps per CTA
            mbar_init(&empty_[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], 2 * 4);  // 4 epilogue warps per CTA
        }
        mbar_init(&mma_done, 1);
        abort_sh = 0;
        fence_mbar_init();
    }
    __syncthreads();
    cluster_sync_all();
    if (warp == 1) {
        tmem_alloc_pair(&tmem_sh, 2 * TMEM_COLS);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;

    if (warp == 0) {
        if (lane == 0) {
            long long kit = 0;
            bool ok = true;
            for (int t = pair; t < ntiles && ok; t += npairs) {
                int fi, rs0, c0;
                gp_tile(P, t, fi, rs0, c0);
                const FamDesc &F = P.b.f[fi];
                if (!rows_active(F, rs0)) continue;
                const int rh = rs0 + (int)rank * TC_M;
                const int NA = F.BP / TC_BK;
                for (int ka = 0; ka < NA; ka += GP_ATOMS, ++kit) {
                    const int na = NA - ka < GP_ATOMS ? NA - ka : GP_ATOMS;
                    const int s = (int)(kit % NST);
                    const long long n = kit / NST;
                    if (n > 0 &&
                        !mbar_wait(&empty_[s], (uint32_t)((n - 1) & 1), &abort_sh, err, ERR_TIMEOUT_TMA)) {
                        ok = false;
                        break;
                    }
                    uint8_t *st = smem + s * GRSTAGE;
                    const uint32_t bar = cluster_addr(&full_[s], 0);
                    if (leader) mbar_expect_tx(&full_[s], 2 * na * 2 * A_BYTES);
                    for (int a = 0; a < na; ++a) {
                        tma_load_2d_pair(st + 2 * a * A_BYTES, &P.dhi[fi], bar, (ka + a) * TC_BK, rh);
                        tma_load_2d_pair(st + (2 * a + 1) * A_BYTES, &P.dlo[fi], bar, (ka + a) * TC_BK, rh);
                    }
                }
            }
            if (leader)
                for (long long k = kit - NST < 0 ? 0 : kit - NST; k < kit; ++k)
                    mbar_drain(&full_[k % NST], (uint32_t)((k / NST) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            const uint32_t idesc = idesc_bf16(2 * TC_M, GRN);
            long long kit = 0;
            int ti = 0;
            bool ok = true;
            for (int t = pair; t < ntiles && ok; t += npairs) {
                int fi, rs0, c0;
                gp_tile(P, t, fi, rs0, c0);
                const FamDesc &F = P.b.f[fi];
                if (!rows_active(F, rs0)) continue;
                const int a = ti & 1, use = ti >> 1;
                if (use > 0 && !mbar_wait(&acc_empty[a], (uint32_t)((use - 1) & 1), &abort_sh, err,
                                          ERR_TIMEOUT_MMA))
                    break;
                tc_fence_after();
                const uint32_t dt = tmem + a * TMEM_COLS;
                const int NA = F.BP / TC_BK;
                for (int ka = 0; ka < NA; ka += GP_ATOMS, ++kit) {
                    const int na = NA - ka < GP_ATOMS ? NA - ka : GP_ATOMS;
                    const int s = (int)(kit % NST);
                    const uint32_t ph = (uint32_t)((kit / NST) & 1);
                    if (!mbar_wait(&full_[s], ph, &abort_sh, err, ERR_TIMEOUT_MMA)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    uint8_t *st = smem + s * GRSTAGE;
                    for (int a2 = 0; a2 < na; ++a2) {
                        const uint32_t ah = smem_u32(st + 2 * a2 * A_BYTES);
                        const uint32_t al = smem_u32(st + (2 * a2 + 1) * A_BYTES);
                        const uint32_t bx = smem_u32(st + B_OFF + a2 * B_BYTES);
#pragma unroll
                        for (int k = 0; k < TC_BK / 16; ++k)
                            mma_bf16_pair(dt, sdesc(ah + 32 * k), sdesc(bx + 32 * k), idesc,
                                          (ka > 0 || a2 > 0 || k > 0) ? 1u : 0u);
#pragma unroll
                        for (int k = 0; k < TC_BK / 16; ++k)
                            mma_bf16_pair(dt, sdesc(al + 32 * k), sdesc(bx + 32 * k), idesc, 1u);
                    }
                    mma_commit_pair(&empty_[s]);
                }
                if (!ok) break;
                mma_commit_pair(&acc_full[a]);
                ++ti;
            }
            mma_commit_pair(&mma_done);  // arrives in both CTAs when every MMA above is complete
        }
    } else if (warp < 2 + GR_PROD / 32) {
        // ---- one-hot X^T producer: thread p writes row p % 128 of this
        // CTA's column half for K atom p / 128 of every stage
        const int p = threadIdx.x - 64;
        const int prow = p % TC_M, pa = p / TC_M;
        long long kit = 0;
        bool ok = true;
        for (int t = pair; t < ntiles && ok; t += npairs) {
            int fi, rs0, c0;
            gp_tile(P, t, fi, rs0, c0);
            const FamDesc &F = P.b.f[fi];
            if (!rows_active(F, rs0)) continue;
            const int BP = F.BP, NA = BP / TC_BK, NQ = F.N * Q;
            const int c = c0 + (int)rank * HN + prow;
            int src_i = 0;
            uint32_t kk = 0xFFu;  // never equals a stored state (0..20, or 0x7F padding)
            if (c < NQ) {
                src_i = c / Q;
                kk = (uint32_t)(c % Q);
            } else if (c == NQ) {
                src_i = F.N;  // the all-ones row of msaT
                kk = 0;
            }
            kk *= 0x01010101u;
            const bool has_row = prow < HN;
            const uint4 *srcT = (const uint4 *)(F.msaT + (size_t)src_i * BP);
            uint4 cur[4], nxt[4];
            {
                const int ka0 = pa < NA ? pa : 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) cur[q] = __ldg(srcT + (size_t)ka0 * (TC_BK / 16) + q);
            }
            for (int ka = 0; ka < NA; ka += GP_ATOMS, ++kit) {
                const int na = NA - ka < GP_ATOMS ? NA - ka : GP_ATOMS;
                const int s = (int)(kit % NST);
                const long long n = kit / NST;
                // the next stage's bytes for this thread's atom
                const int kn = ka + GP_ATOMS + pa < NA ? ka + GP_ATOMS + pa
                                                       : (ka + pa < NA ? ka + pa : 0);
#pragma unroll
                for (int q = 0; q < 4; ++q) nxt[q] = __ldg(srcT + (size_t)kn * (TC_BK / 16) + q);
                const bool got = n == 0 || mbar_wait(&empty_[s], (uint32_t)((n - 1) & 1), &abort_sh,
                                                     err, ERR_TIMEOUT_PROD);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                if (has_row && pa < na) {
                    uint8_t *bt = smem + s * GRSTAGE + B_OFF + pa * B_BYTES;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {  // 16 sequences per word group
                        const uint4 x = cur[q];
                        const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
                        uint32_t o[8];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const uint32_t m = __vcmpeq4(xs[u], kk);
                            o[2 * u] = __byte_perm(m, 0, 0x1100) & 0x3F803F80u;
                            o[2 * u + 1] = __byte_perm(m, 0, 0x3322) & 0x3F803F80u;
                        }
                        *(uint4 *)(bt + swz(prow, 2 * q)) = make_uint4(o[0], o[1], o[2], o[3]);
                        *(uint4 *)(bt + swz(prow, 2 * q + 1)) = make_uint4(o[4], o[5], o[6], o[7]);
                    }
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(cluster_addr(&full_[s], 0));
#pragma unroll
                for (int q = 0; q < 4; ++q) cur[q] = nxt[q];
            }
        }
    } else {
        // ---- epilogue: one row of this CTA's 128 per thread (its tensor-
        // memory lane), 16 columns at a time: 2 lambda Theta added, the
        // diagonal block, the padding rows and columns zeroed, G written
        const int q4 = warp & 3;
        const int er = q4 * 32 + lane;
        int ti = 0;
        for (int t = pair; t < ntiles; t += npairs) {
            int fi, rs0, c0;
            gp_tile(P, t, fi, rs0, c0);
            const FamDesc &F = P.b.f[fi];
            if (!rows_active(F, rs0)) continue;
            const int a = ti & 1, use = ti >> 1;
            const int row = rs0 + (int)rank * TC_M + er;
            const int KP = F.KP, NQ = F.N * Q;
            const bool live_row = row < F.R;
            const int r = row / QP, sstate = row % QP;
            const float *th = F.theta + (size_t)(live_row ? row : 0) * KP;
            float *g = F.G + (size_t)(live_row ? row : 0) * KP;
            const bool ok = mbar_wait(&acc_full[a], (uint32_t)(use & 1), &abort_sh, err, ERR_TIMEOUT_EPI);
            tc_fence_after();
            const uint32_t tl = tmem + a * TMEM_COLS + ((uint32_t)(q4 * 32) << 16);
            for (int cc = 0; cc < GRN / 16; ++cc) {
                float v[16];
                tmem_ld16(tl + cc * 16, v);
                tmem_wait_ld();
                const int cb = c0 + cc * 16;
                if (ok && live_row && cb < KP) {  // KP is a multiple of 64
                    float4 tv[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) tv[q] = *(const float4 *)(th + cb + 4 * q);
                    float o[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int cu = cb + u;
                        const float tu = (&tv[u >> 2].x)[u & 3];
                        float val;
                        if (sstate >= Q || cu > NQ || (cu >= r * Q && cu < r * Q + Q)) val = 0.0f;
                        else if (cu == NQ) val = v[u] + two_lh * tu;
                        else val = v[u] + two_lj * tu;
                        o[u] = val;
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        *(float4 *)(g + cb + 4 * q) =
                            make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
                }
                __syncwarp();
            }
            // this warp's tensor-memory reads of the tile are done
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(cluster_addr(&acc_empty[a], 0));
            ++ti;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1 && lane == 0) mbar_drain(&mma_done, 0);  // every MMA into this CTA's memory
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, 2 * TMEM_COLS);
    }
    cluster_sync_all();
}

// ---------------------------------------------------------------- self-test
// The bounded wait of the pipelines above on a barrier that nothing
// arrives on: it gives up after its cycle budget, raises the CTA's abort
// flag and records ERR_TIMEOUT_SELFTEST in the error word, and the kernel
// returns normally (no fault, the context stays usable).
__global__ void k_wait_selftest(int *__restrict__ err)
{
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_sh;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_sh = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&bar, 0, &abort_sh, err, ERR_TIMEOUT_SELFTEST);
    __syncthreads();
}

// ---------------------------------------------------------------- helpers
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

// msaT[i][b] = S[b][i] (b < B), 0x7F beyond B; row N is the constant-feature
// row (0 for b < B, 0x7F beyond)
__global__ void k_msa_transpose(const int8_t *__restrict__ msa, int B, int N, int BP,
                                int8_t *__restrict__ msaT)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)(N + 1) * BP;
    if (idx >= total) return;
    int i = (int)(idx / BP), b = (int)(idx % BP);
    int8_t v = 0x7F;
    if (b < B) v = (i < N) ? msa[(size_t)b * N + i] : 0;
    msaT[idx] = v;
}

// f_data[r] = -(sum over sequence tiles of the partials) / B_eff, per family
__global__ void k_tc_finish(const __grid_constant__ TcBatch b)
{
    const FamDesc &F = b.f[blockIdx.x];
    const int nbt = F.BP / TC_M;
    for (int r = threadIdx.x; r < F.N; r += blockDim.x) {
        if (F.active && !F.active[r]) continue;  // not evaluated: keep its value
        double t = 0.0;
        for (int y = 0; y < nbt; ++y) t += F.partial[(size_t)y * F.N + r];
        F.f_data[r] = -t / F.beff;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    // looked up once per process (a function-local static is initialised
    // exactly once, whichever thread gets here first)
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000)p;
        return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }();
    return fn;
}

// 3-D bf16 map over a site-major [N][QP][KP] array (the split Theta, or the
// residual D^T with KP = BP) that skips the padding rows: dims (KP, Q
// states, N sites), box (64, Q, sh) lands as sh x Q rows of 128 bytes,
// 128-byte swizzled
bool make_map_sites(CUtensorMap *m, const void *base, uint64_t KP, uint64_t N, uint32_t sh)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {KP, (cuuint64_t)Q, N};
    cuuint64_t strides[2] = {KP * 2, (cuuint64_t)QP * KP * 2};
    cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)Q, sh};
    cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides,
              box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// 2D bf16 map over a row-major [outer][inner] array, 128-byte swizzled boxes
bool make_map(CUtensorMap *m, const void *base, uint64_t inner, uint64_t outer,
              uint32_t box_inner, uint32_t box_outer)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides,
              box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

int tc_padded_B(int B) { return (B + TC_M - 1) / TC_M * TC_M; }

cudaError_t launch_wait_selftest(int *err, cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(err);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_split_theta(const float *theta, size_t n, __nv_bfloat16 *hi,
                               __nv_bfloat16 *lo, cudaStream_t st)
{
    k_split<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(theta, n, hi, lo);
    count_launches(1);
    return cudaGetLastError();
}

// one family's scratch: D^T hi | D^T lo | partial | msaT
size_t tc_family_scratch_bytes(int B, int N)
{
    const size_t BP = tc_padded_B(B), R = (size_t)N * QP;
    const size_t nbt = BP / TC_M;
    return 2 * align256(R * BP * 2) + align256(nbt * N * sizeof(double)) +
           align256((size_t)(N + 1) * BP);
}

int tc_supported()
{
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    return (major == 10 && minor == 3 && encode_fn() != nullptr) ? 1 : 0;
}

cudaError_t launch_tc_prepare(TcBatch &b, void *const *scratch, cudaStream_t st)
{
    for (int i = 0; i < b.nfam; ++i) {
        FamDesc &F = b.f[i];
        F.BP = tc_padded_B(F.B);
        F.R = F.N * QP;
        F.KP = (F.N * Q + 1 + KALIGN - 1) / KALIGN * KALIGN;
        const size_t nbt = F.BP / TC_M;
        char *p = (char *)scratch[i];
        F.dt_hi = (__nv_bfloat16 *)p;
        p += align256((size_t)F.R * F.BP * 2);
        F.dt_lo = (__nv_bfloat16 *)p;
        p += align256((size_t)F.R * F.BP * 2);
        F.partial = (double *)p;
        p += align256(nbt * F.N * sizeof(double));
        int8_t *msaT = (int8_t *)p;
        F.msaT = msaT;
        const size_t nT = (size_t)(F.N + 1) * F.BP;
        k_msa_transpose<<<(unsigned)((nT + 255) / 256), 256, 0, st>>>(F.msa, F.B, F.N, F.BP, msaT);
        count_launches(1);
    }
    return cudaGetLastError();
}


int tc_stages(int stage_bytes, int slab_bytes)
{
    int n = (SMEM_BUDGET - slab_bytes) / stage_bytes;
    return n > MAX_STAGES ? MAX_STAGES : n;
}

int num_sms()
{
    static std::atomic<int> cache[64];  // per device; 0 = not queried yet
    int dev = 0;
    cudaGetDevice(&dev);
    std::atomic<int> &c = cache[dev & 63];
    int n = c.load();
    if (!n) {
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
        c.store(n);
    }
    return n;
}

bool tc_config_valid(const TcConfig &c)
{
    const bool lg = c.lg_pair ? ((c.lg_pair == 1 || c.lg_pair == 2) &&
                                 (c.lg_sites == 4 || c.lg_sites == 8 || c.lg_sites == 10 ||
                                  c.lg_sites == 12))
                              : (c.lg_sites >= 2 && c.lg_sites <= MAX_LG_SITES && c.lg_sites % 2 == 0);
    // one CTA: widths in steps of 16 (the MMA's N); a pair splits the width in two halves
    return lg && c.gr_ncols >= 32 && c.gr_ncols <= 256 && c.gr_ncols % (c.gr_pair ? 32 : 16) == 0 &&
           (c.gr_rows == TC_M || c.gr_rows == 2 * TC_M) &&
           (c.gr_pair == 0 || (c.gr_pair == 1 && c.gr_rows == 2 * TC_M));
}

cudaError_t launch_grad_pair(const GradParams &gp, int ntiles, float two_lh, float two_lj, int *err,
                             cudaStream_t st)
{
    static std::atomic<unsigned long long> attr{0};
    const int smem = gp.stages * gp.stage_bytes + 1024;
    // the limit is raised once per device, to the largest any column width uses
    cudaError_t e = set_smem_limit_once((const void *)k_tc_grad_pair, SMEM_BUDGET + 1024, attr);
    if (e) return e;
    if (ntiles <= 0) return cudaSuccess;
    // persistent: as many clusters as fit at once (one CTA per SM)
    const int clusters = std::min(ntiles, num_sms() / 2);
    cudaLaunchConfig_t lc = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.gridDim = dim3(2 * clusters);
    lc.blockDim = dim3(GP_THREADS);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, k_tc_grad_pair, gp, two_lh, two_lj, err);
}

// resident 2-CTA clusters of the pair kernel on this device (cached)
template <int SH, int ATOMS>
int pair_clusters(int smem)
{
    static std::atomic<int> cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    std::atomic<int> &c = cache[dev & 63];
    int n = c.load();
    if (!n) {
        cudaLaunchConfig_t lc = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.gridDim = dim3(2 * 256);
        lc.blockDim = dim3(LP_THREADS);
        lc.dynamicSmemBytes = smem;
        lc.attrs = at;
        lc.numAttrs = 1;
        if (cudaOccupancyMaxActiveClusters(&n, k_tc_logits_pair<SH, ATOMS>, &lc) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = num_sms() / 2;
        }
        c.store(n);
    }
    return n;
}

template <int SH, int ATOMS>
cudaError_t launch_logits_pair(PairParams &pp, int ntiles, int *err, cudaStream_t st)
{
    static std::atomic<unsigned long long> attr{0};
    pp.stage_bytes = PairShape<SH, ATOMS>::STAGE;
    pp.stages = tc_stages(pp.stage_bytes, 0);
    const int smem = pp.stages * pp.stage_bytes + 1024;
    cudaError_t e = set_smem_limit_once((const void *)k_tc_logits_pair<SH, ATOMS>, SMEM_BUDGET + 1024,
                                        attr);
    if (e) return e;
    const int clusters = std::min(ntiles, pair_clusters<SH, ATOMS>(smem));
    if (clusters <= 0) return cudaSuccess;
    cudaLaunchConfig_t lc = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.gridDim = dim3(2 * clusters);
    lc.blockDim = dim3(LP_THREADS);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, k_tc_logits_pair<SH, ATOMS>, (const PairParams)pp, err);
}

cudaError_t launch_tc_eval(void *prof, const TcBatch &b_in, const TcConfig &cfg, double lambda_h,
                           double lambda_Jp, int *err, cudaStream_t st, int which)
{
    static std::atomic<unsigned long long> attr_lg{0}, attr_gr{0};
    cudaError_t e = set_smem_limit_once((const void *)k_tc_logits, SMEM_BUDGET + 1024, attr_lg);
    if (e) return e;
    e = set_smem_limit_once((const void *)k_tc_grad, SMEM_BUDGET + 1024, attr_gr);
    if (e) return e;
    if (b_in.nfam < 1 || b_in.nfam > MAX_FAM || !tc_config_valid(cfg))
        return cudaErrorInvalidValue;
    // large parameter blocks, built on the host and passed by value (a launch
    // copies them), one pair per host thread so that contexts driven from
    // different threads do not share them
    thread_local LogitsParams lp;
    thread_local GradParams gp;
    thread_local PairParams pp;
    lp.b = b_in;
    const int lg_ncols = cfg.lg_sites * QP;
    int tl = 0, tg = 0;
    for (int i = 0; i < lp.b.nfam; ++i) {
        FamDesc &F = lp.b.f[i];
        F.tile0_logits = tl;
        F.tile0_grad = tg;
        const int nbt = cfg.lg_pair ? (F.BP / TC_M + 1) / 2 : F.BP / TC_M;
        tl += nbt * ((F.N + cfg.lg_sites - 1) / cfg.lg_sites);
        // row tiles: padded rows on CTA pairs, GR_SITES sites per 128 rows on one CTA
        const int nrt = cfg.gr_pair ? (F.R + cfg.gr_rows - 1) / cfg.gr_rows
                                    : (F.N + GR_SITES * cfg.gr_rows / TC_M - 1) /
                                          (GR_SITES * cfg.gr_rows / TC_M);
        tg += ((F.KP + cfg.gr_ncols - 1) / cfg.gr_ncols) * nrt;
    }
    lp.b.ntiles_logits = tl;
    lp.b.ntiles_grad = tg;
    gp.b = lp.b;
    lp.sites = cfg.lg_sites;
    lp.ncols = lg_ncols;
    lp.stage_bytes = LG_A_BYTES + 2 * lg_ncols * TC_BK * 2;
    lp.stages = tc_stages(lp.stage_bytes, 0);
    gp.rows = cfg.gr_rows;
    gp.ncols = cfg.gr_ncols;
    if (cfg.gr_pair)  // two K atoms per stage: D^T hi/lo of 128 rows and half the columns each
        gp.stage_bytes = GP_ATOMS * (2 * GR_A_BYTES + (cfg.gr_ncols / 2) * TC_BK * 2);
    else
        gp.stage_bytes = 2 * (cfg.gr_rows / TC_M) * GR_A_BYTES + cfg.gr_ncols * TC_BK * 2;
    gp.stages = tc_stages(gp.stage_bytes, 0);
    const int sh = cfg.lg_sites / 2;
    for (int i = 0; i < lp.b.nfam; ++i) {
        const FamDesc &F = lp.b.f[i];
        const bool lg_ok =
            cfg.lg_pair ? (make_map_sites(&pp.hi[i], F.th_hi, F.KP, F.N, sh) &&
                           make_map_sites(&pp.lo[i], F.th_lo, F.KP, F.N, sh))
                        : (make_map(&lp.hi[i], F.th_hi, F.KP, F.R, TC_BK, lg_ncols) &&
                           make_map(&lp.lo[i], F.th_lo, F.KP, F.R, TC_BK, lg_ncols));
        // a pair's CTA loads 128 padded rows; one CTA loads GR_SITES sites per box
        const bool gr_ok =
            cfg.gr_pair ? (make_map(&gp.dhi[i], F.dt_hi, F.BP, F.R, TC_BK, TC_M) &&
                           make_map(&gp.dlo[i], F.dt_lo, F.BP, F.R, TC_BK, TC_M))
                        : (make_map_sites(&gp.dhi[i], F.dt_hi, F.BP, F.N, GR_SITES) &&
                           make_map_sites(&gp.dlo[i], F.dt_lo, F.BP, F.N, GR_SITES));
        if (!lg_ok || !gr_ok) return cudaErrorInvalidValue;
    }
    if (which & 1) {
        void *t0 = prof ? prof_start(prof) : nullptr;
        if (cfg.lg_pair) {
            pp.b = lp.b;
            cudaError_t e2 = cudaSuccess;
            // lg_pair 1: stages of two K atoms; 2: stages of one atom (more stages)
            if (sh == 2) e2 = cfg.lg_pair == 2 ? launch_logits_pair<2, 1>(pp, tl, err, st)
                                               : launch_logits_pair<2, 2>(pp, tl, err, st);
            else if (sh == 4) e2 = cfg.lg_pair == 2 ? launch_logits_pair<4, 1>(pp, tl, err, st)
                                                    : launch_logits_pair<4, 2>(pp, tl, err, st);
            else if (sh == 5) e2 = cfg.lg_pair == 2 ? launch_logits_pair<5, 1>(pp, tl, err, st)
                                                    : launch_logits_pair<5, 2>(pp, tl, err, st);
            else e2 = cfg.lg_pair == 2 ? launch_logits_pair<6, 1>(pp, tl, err, st)
                                       : launch_logits_pair<6, 2>(pp, tl, err, st);
            if (e2) return e2;
        } else {
            const int grid = std::min(tl, num_sms());
            if (grid > 0)
                k_tc_logits<<<grid, LG_THREADS, lp.stages * lp.stage_bytes + 1024, st>>>(lp, err);
        }
        if (prof) prof_stop(prof, "tc_logits", t0);
        k_tc_finish<<<lp.b.nfam, 128, 0, st>>>(lp.b);
        count_launches(2);
    }
    if (which & 2) {
        void *t1 = prof ? prof_start(prof) : nullptr;
        if (cfg.gr_pair) {
            cudaError_t e3 = launch_grad_pair(gp, tg, (float)(2.0 * lambda_h),
                                              (float)(2.0 * lambda_Jp), err, st);
            if (e3) return e3;
        } else if (tg > 0) {
            k_tc_grad<<<tg, GR_THREADS, gp.stages * gp.stage_bytes + 1024, st>>>(
                gp, (float)(2.0 * lambda_h), (float)(2.0 * lambda_Jp), err);
        }
        if (prof) prof_stop(prof, "tc_grad", t1);
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace plm
