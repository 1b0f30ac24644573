// k_lbfgs.cu -- batched per-site L-BFGS for step 3 of the rundown.
//
// Every site r minimises its own g_r^(reg) (Eq. g_regdef2) over the row
// block Theta[r] (Eq. npll_2: the N problems are independent); the paper
// names limited-memory BFGS as the minimiser (Sec. 5) and starts at the
// origin (Sec. 6).  All sites share each objective+gradient evaluation; a
// site keeps its own curvature pairs, step length and stopping state.
//
// Vectors are FP32.  Inner products are accumulated per thread in
// double-float (FP32 arithmetic, ~44 significant bits; each float4's four
// products summed by FMAs, then added without error), then reduced across threads and chunks in FP64; every scalar of the
// recursion and of the line search is FP64.  Each site's segment is cut
// into chunks; one CTA per (chunk, site) streams the vectors and writes
// partial sums, and a one-warp-per-site kernel reduces them in a fixed
// order and does the scalar work, so results do not depend on scheduling.
//
// Direction: the compact representation of the L-BFGS inverse Hessian
// (Byrd, Nocedal & Schnabel 1994; Nocedal & Wright Eq. 7.24) with
// H0 = gamma I, gamma = s'y / y'y of the newest pair:
//     H g = gamma g + S p - gamma Y R^{-1} u,
//     u = S'g, v = Y'g, p = R^{-T} ((D + gamma Y'Y) R^{-1} u - gamma v),
// R the upper triangle of S'Y (age order), D its diagonal.  u and v are
// kept current incrementally: when the accepted step adds the pair
// (s_n, y_n) and moves g to g + y_n, u_j += s_j'y_n and v_j += y_j'y_n for
// the older pairs, and u_n = s_n'g_new, v_n = y_n'g_old + y_n'y_n for the new
// one (the commit pass forms s_n'g_new and y_n'g_old from values it already
// holds).  So one streaming pass forms S'y_n and Y'y_n (which also keep S'Y
// and Y'Y current) and a second pass forms d.  The result equals the
// two-loop recursion's.
//
// Step: strong-Wolfe search (c1, c2) in the style of Nocedal & Wright
// Alg. 3.5/3.6, driven by the directional derivative: the objective is
// convex, so phi'(alpha) is nondecreasing and brackets the minimiser along
// the line even where FP32 rounding makes differences of f unresolvable.
// Sufficient decrease allows a noise band `noise * max(1, |f0|)` on f, or
// is certified by phi'(alpha) <= c1 phi'(0) (convexity).
#include <map>
#include <mutex>
#include <utility>

#include "plm_device.cuh"
#include "plm_internal.cuh"

namespace plm {

namespace {

constexpr int LB_THREADS = 128;

// sum K per-thread double-float values over the block (fixed order) and
// write them as FP64: a butterfly of error-free FP32 pair additions inside
// each warp, then one thread per value adds the warps' pairs in FP64.  The
// block's threads all take part; the shared buffer is free again on return.
template <int K>
__device__ __forceinline__ void block_write(DF (&v)[K], double *out)
{
    __shared__ float rh[LB_THREADS / 32][K], rl[LB_THREADS / 32][K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float hi = v[k].hi, lo = v[k].lo;
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
        if (lane == 0) {
            rh[wid][k] = hi;
            rl[wid][k] = lo;
        }
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double t = 0.0;
        for (int w = 0; w < LB_THREADS / 32; ++w)
            t += (double)rh[w][threadIdx.x] + (double)rl[w][threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

// fixed-order sum over the chunks of one site (one warp): returns the
// total of slot k of the site's partial records
__device__ __forceinline__ double chunk_sum(const double *part, const SiteInfo &si, int k)
{
    const int lane = threadIdx.x & 31;
    double t = 0.0;
    for (int c = lane; c < si.nchunks; c += 32) t += part[(size_t)(si.chunk0 + c) * LB_PART + k];
    return warp_sum_d(t);
}

// the same total for one slot, summed by a single thread in chunk order (a
// warp sums several slots at once this way)
__device__ __forceinline__ double lane_chunk_sum(const double *part, const SiteInfo &si, int k)
{
    const double *q = part + (size_t)si.chunk0 * LB_PART + k;
    double t = 0.0;
    // unrolled so that the independent loads are in flight together; the
    // additions keep the chunk order
#pragma unroll 8
    for (int c = 0; c < si.nchunks; ++c) t += q[(size_t)c * LB_PART];
    return t;
}

// Above this many chunks (a site of a very large problem, or the single
// problem of the symmetric solve with all parameters) a thread per slot
// walking every chunk record is bound by load latency; such a site's slots
// are summed by the whole warp instead (warp_chunk_sums).  Sites at or below
// it keep the per-thread chunk order.
constexpr int LB_WARP_SUM_MIN = 64;

// totals of the K slots slot[0..K) of one site: the lanes take alternate
// chunks and accumulate every slot of each chunk record they read (all loads
// independent), then a fixed-order butterfly; every lane gets the totals
template <int K>
__device__ __forceinline__ void warp_chunk_sums(const double *part, const SiteInfo &si,
                                                const int (&slot)[K], double (&t)[K])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; ++k) t[k] = 0.0;
    for (int c = lane; c < si.nchunks; c += 32) {
        const double *q = part + (size_t)(si.chunk0 + c) * LB_PART;
#pragma unroll
        for (int k = 0; k < K; ++k) t[k] += q[slot[k]];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) t[k] = warp_sum_d(t[k]);
}

struct Chunk {
    size_t base4, e0, e1;
    int site;
};

__device__ __forceinline__ Chunk chunk_at(const SiteInfo *si, const ChunkInfo *ci, int c)
{
    const ChunkInfo x = ci[c];
    Chunk ch;
    ch.site = x.site;
    ch.base4 = (size_t)si[x.site].off4;
    ch.e0 = (size_t)x.e0;
    ch.e1 = (size_t)x.e1;
    return ch;
}

__device__ __forceinline__ double *part_rec(double *part, int c)
{
    return part + (size_t)c * LB_PART;
}

__device__ __forceinline__ float4 f4z() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// ------------------------------------------------------------ start
__global__ void __launch_bounds__(LB_THREADS)
k_init_dots(const float *__restrict__ g, const SiteInfo *si, const ChunkInfo *ci, int c0, int c1,
            double *part)
{
    for (int c = c0 + blockIdx.x; c < c1; c += gridDim.x) {
        const Chunk ch = chunk_at(si, ci, c);
        const float4 *g4 = (const float4 *)g + ch.base4;
        DF acc[1];
        for (size_t e = ch.e0 + threadIdx.x; e < ch.e1; e += LB_THREADS) {
            const float4 gv = g4[e];
            df_dot4(acc[0], gv, gv);
        }
        block_write<1>(acc, part_rec(part, c));
    }
}

__global__ void k_init_finish(SiteState *ss, const double *__restrict__ f, const double *part,
                              const SiteInfo *si, int s0, SolveParams p)
{
    const int r = s0 + blockIdx.x;
    const double gg = chunk_sum(part, si[r], 0);
    if (threadIdx.x != 0) return;
    SiteState &s = ss[r];
    s.f = f[r];
    s.gnorm2 = gg;
    s.hist = 0;
    s.head = 0;
    s.iters = 0;
    s.trials = 0;
    s.phase = 0;
    s.gamma = 1.0;
    s.commit_round = -1;
    s.commit_slot = 0;
    for (int i = 0; i < MAX_M; ++i)
        for (int j = 0; j < MAX_M; ++j) {
            s.SY[i][j] = 0.0;
            s.YY[i][j] = 0.0;
        }
    s.status = (sqrt(gg) <= p.gtol) ? SITE_CONVERGED
               : (p.max_iter <= 0 ? SITE_FAILED : SITE_READY);
}

// ------------------------------------------------------------ direction
__device__ __forceinline__ bool slot_valid(int j, int head, int hist, int M)
{
    return ((head - 1 - j + 2 * M) % M) < hist;  // distance from the newest slot
}

// squares of theta_t into the penalty sums (field column separately) and
// its bf16 hi/lo split for the tensor-core evaluation
__device__ __forceinline__ void trial_penalty_split(const float4 x, size_t e, size_t base4, int NQ,
                                                    int KP, __nv_bfloat16 *__restrict__ hi,
                                                    __nv_bfloat16 *__restrict__ lo, DF &pj,
                                                    DF &ph)
{
    const float xv[4] = {x.x, x.y, x.z, x.w};
    // 32-bit arithmetic: 4 e stays below 2^32 for every segment this solver
    // streams (at most N QP KP elements)
    const int c0 = (int)((4u * (uint32_t)e) % (uint32_t)KP);
    float sj = 0.0f, sh = 0.0f;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        if (c0 + u == NQ) sh = fmaf(xv[u], xv[u], sh);
        else sj = fmaf(xv[u], xv[u], sj);
    }
    df_add(pj, sj);
    df_add(ph, sh);
    if (hi) {
        const size_t at = 4 * (base4 + e);
        __align__(8) __nv_bfloat16 h4[4], l4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            h4[u] = __float2bfloat16_rn(xv[u]);
            l4[u] = __float2bfloat16_rn(xv[u] - __bfloat162float(h4[u]));
        }
        *(uint2 *)(hi + at) = *(const uint2 *)h4;
        *(uint2 *)(lo + at) = *(const uint2 *)l4;
    }
}

// the small FP64 algebra of the compact form, one warp per site (the site's
// matrices are staged in shared memory)
template <int M>
__global__ void k_dir_solve(SiteState *ss, const double *part, const SiteInfo *si, int s0,
                            int *round_ptr, int *counters)
{
    const int r = s0 + blockIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // start of a round: advance the round counter; keep the number of
        // searches that continue from the last round (the trial pass exits
        // at once when there are none) and clear this round's counts
        *round_ptr += 1;
        counters[2] = counters[0];
        counters[0] = 0;
        counters[1] = 0;
    }
    SiteState &s = ss[r];
    if (s.status != SITE_READY) return;
    __shared__ double tot[2 * M + 2];
    __shared__ double SY[M][M], YY[M][M];
    const int hist = s.hist, head = s.head;
    const int lane = threadIdx.x;
    if (hist > 0) {
        // slots 0..2M-1: S'y_n, Y'y_n; then s_n'g_new and y_n'g_old
        if (si[r].nchunks > LB_WARP_SUM_MIN) {
            int slot[2 * M + 2];
            double t[2 * M + 2];
#pragma unroll
            for (int k = 0; k < 2 * M + 2; ++k)
                slot[k] = k < 2 * M ? k : (k == 2 * M ? LB_SLOT_SG : LB_SLOT_YG);
            warp_chunk_sums(part, si[r], slot, t);
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < 2 * M + 2; ++k) tot[k] = t[k];
        } else if (lane < 2 * M + 2) {
            const int k = lane < 2 * M ? lane : (lane == 2 * M ? LB_SLOT_SG : LB_SLOT_YG);
            tot[lane] = lane_chunk_sum(part, si[r], k);
        }
        for (int k = lane; k < M * M; k += 32) {
            SY[k / M][k % M] = s.SY[k / M][k % M];
            YY[k / M][k % M] = s.YY[k / M][k % M];
        }
    }
    __syncwarp();
    if (lane != 0) return;
    for (int j = 0; j < MAX_M; ++j) s.cs[j] = s.cy[j] = 0.0;
    s.cg = 1.0;
    // first trial step: 1/||g|| on the very first (steepest-descent) step, else 1
    s.alpha = (s.iters == 0) ? 1.0 / sqrt(s.gnorm2) : 1.0;
    if (hist == 0) return;
    const int n = (head - 1 + M) % M;
    // new column of S'Y and row/column of Y'Y; u, v moved to g_new
    for (int j = 0; j < M; ++j) {
        if (!slot_valid(j, head, hist, M)) continue;
        SY[j][n] = tot[j];
        YY[j][n] = tot[M + j];
        YY[n][j] = tot[M + j];
        if (j != n) {
            s.u[j] += tot[j];
            s.v[j] += tot[M + j];
        }
    }
    s.u[n] = tot[2 * M];
    s.v[n] = tot[2 * M + 1] + YY[n][n];
    for (int j = 0; j < M; ++j) {
        if (!slot_valid(j, head, hist, M)) continue;
        s.SY[j][n] = SY[j][n];
        s.YY[j][n] = YY[j][n];
        s.YY[n][j] = YY[n][j];
    }
    if (!(SY[n][n] > 0.0) || !(YY[n][n] > 0.0)) {
        // newest pair violates the curvature condition: restart from -g
        s.hist = 0;
        s.head = 0;
        return;
    }
    s.alpha = 1.0;
    const double gamma = SY[n][n] / YY[n][n];
    int idx[M];
    double u[M], v[M], t1[M], t2[M], pp[M];
    for (int a = 0; a < hist; ++a) {
        idx[a] = (head - hist + a + 2 * M) % M;  // oldest first
        u[a] = s.u[idx[a]];
        v[a] = s.v[idx[a]];
    }
    // t1 = R^{-1} u, R[a][b] = s_a . y_b (a <= b in age order)
    for (int a = hist - 1; a >= 0; --a) {
        double x = u[a];
        for (int b = a + 1; b < hist; ++b) x -= SY[idx[a]][idx[b]] * t1[b];
        t1[a] = x / SY[idx[a]][idx[a]];
    }
    // t2 = (D + gamma Y'Y) t1 - gamma v
    for (int a = 0; a < hist; ++a) {
        double x = SY[idx[a]][idx[a]] * t1[a] - gamma * v[a];
        for (int b = 0; b < hist; ++b) x += gamma * YY[idx[a]][idx[b]] * t1[b];
        t2[a] = x;
    }
    // p = R^{-T} t2
    for (int a = 0; a < hist; ++a) {
        double x = t2[a];
        for (int b = 0; b < a; ++b) x -= SY[idx[b]][idx[a]] * pp[b];
        pp[a] = x / SY[idx[a]][idx[a]];
    }
    s.gamma = gamma;
    s.cg = gamma;
    for (int a = 0; a < hist; ++a) {
        s.cs[idx[a]] = pp[a];
        s.cy[idx[a]] = -gamma * t1[a];
    }
}

// d = -(cg g + sum cs_j s_j + sum cy_j y_j) and, in the same pass, the
// first trial point theta_t = theta + alpha d (with its bf16 split) of the
// new line search.  Partials: slots 0, 1 the penalty sums of theta_t
// (couplings, fields), slot 2 g.d.  Every vector an element needs is loaded
// before any arithmetic.
template <int M>
__global__ void __launch_bounds__(LB_THREADS, 3)
k_dir_apply(const SiteState *ss, const float *__restrict__ g, const float *__restrict__ S,
            const float *__restrict__ Y, float *__restrict__ dir, const float *__restrict__ theta,
            float *__restrict__ theta_t, __nv_bfloat16 *__restrict__ hi,
            __nv_bfloat16 *__restrict__ lo, const SiteInfo *si, const ChunkInfo *ci, int c0, int c1,
            long long vec4, double *part)
{
    for (int c = c0 + blockIdx.x; c < c1; c += gridDim.x) {
        const Chunk ch = chunk_at(si, ci, c);
        const SiteState &s = ss[ch.site];
        if (s.status != SITE_READY) continue;
        const int hist = s.hist, head = s.head;
        const int NQ = si[ch.site].NQ, KP = si[ch.site].KP;
        const float4 *g4 = (const float4 *)g + ch.base4;
        const float4 *S4 = (const float4 *)S + ch.base4;
        const float4 *Y4 = (const float4 *)Y + ch.base4;
        const float4 *t4 = (const float4 *)theta + ch.base4;
        float4 *d4 = (float4 *)dir + ch.base4;
        float4 *o4 = (float4 *)theta_t + ch.base4;
        const float cg = (float)s.cg, al = (float)s.alpha;
        bool valid[M];
        float cs[M], cy[M];
#pragma unroll
        for (int j = 0; j < M; ++j) {
            valid[j] = slot_valid(j, head, hist, M);
            cs[j] = (float)s.cs[j];
            cy[j] = (float)s.cy[j];
        }
        DF acc[3];
        auto apply = [&](size_t e, const float4 &gv, const float4 &tv, const float4 (&sv)[M],
                         const float4 (&yv)[M]) {
            float4 a = make_float4(cg * gv.x, cg * gv.y, cg * gv.z, cg * gv.w);
#pragma unroll
            for (int j = 0; j < M; ++j) {
                a.x += cs[j] * sv[j].x + cy[j] * yv[j].x;
                a.y += cs[j] * sv[j].y + cy[j] * yv[j].y;
                a.z += cs[j] * sv[j].z + cy[j] * yv[j].z;
                a.w += cs[j] * sv[j].w + cy[j] * yv[j].w;
            }
            const float4 dv = make_float4(-a.x, -a.y, -a.z, -a.w);
            d4[e] = dv;
            df_dot4(acc[2], gv, dv);
            const float4 x = make_float4(fmaf(al, dv.x, tv.x), fmaf(al, dv.y, tv.y),
                                         fmaf(al, dv.z, tv.z), fmaf(al, dv.w, tv.w));
            o4[e] = x;
            trial_penalty_split(x, e, ch.base4, NQ, KP, hi, lo, acc[0], acc[1]);
        };
        // two elements per thread and iteration, all their loads issued
        // before any arithmetic (twice the bytes in flight); the elements
        // are applied and accumulated in index order, as one at a time
        for (size_t e = ch.e0 + threadIdx.x; e < ch.e1; e += 2 * LB_THREADS) {
            const size_t e2 = e + LB_THREADS;
            const bool two = e2 < ch.e1;
            const float4 gv = g4[e], tv = t4[e];
            const float4 gv2 = two ? g4[e2] : f4z(), tv2 = two ? t4[e2] : f4z();
            float4 sv[M], yv[M], sv2[M], yv2[M];
#pragma unroll
            for (int j = 0; j < M; ++j) {
                sv[j] = valid[j] ? S4[(size_t)j * vec4 + e] : f4z();
                yv[j] = valid[j] ? Y4[(size_t)j * vec4 + e] : f4z();
                sv2[j] = (valid[j] && two) ? S4[(size_t)j * vec4 + e2] : f4z();
                yv2[j] = (valid[j] && two) ? Y4[(size_t)j * vec4 + e2] : f4z();
            }
            apply(e, gv, tv, sv, yv);
            if (two) apply(e2, gv2, tv2, sv2, yv2);
        }
        block_write<3>(acc, part_rec(part, c));
    }
}

// line-search set-up.  A direction that is not a descent direction
// (rounding in FP32) drops the history: the site stays READY and takes the
// steepest-descent direction in the next round (its trial point of this
// round is not evaluated).
__global__ void k_dir_finish(SiteState *ss, const double *part, const SiteInfo *si, int s0,
                             uint8_t *active)
{
    const int r = s0 + blockIdx.x;
    SiteState &s = ss[r];
    if (s.status == SITE_READY) {
        const double dg0 = chunk_sum(part, si[r], 2);
        if (threadIdx.x == 0) {
            if (!(dg0 < 0.0)) {
                if (s.hist == 0) s.status = SITE_FAILED;  // -g itself is not a descent direction
                s.hist = 0;
                s.head = 0;
            } else {
                s.f0 = s.f;
                s.dg0 = dg0;
                s.a_prev = 0.0;
                s.f_prev = s.f;
                s.dg_prev = dg0;
                s.a_lo = 0.0;
                s.f_lo = s.f;
                s.dg_lo = dg0;
                s.a_hi = 0.0;
                s.f_hi = 0.0;
                s.dg_hi = 0.0;
                s.phase = 0;
                s.trials = 0;
                s.status = SITE_SEARCHING;
            }
        }
    }
    // the sites this round evaluates
    if (threadIdx.x == 0) active[r] = s.status == SITE_SEARCHING ? 1 : 0;
}

// ------------------------------------------------------------ line search
// later trial points of a line search: theta_t = theta + alpha d (and its
// bf16 split); penalty partials in slots 0, 1.  (The first trial point of
// each search is formed with the direction.)
__global__ void __launch_bounds__(LB_THREADS)
k_trial(const SiteState *ss, const float *__restrict__ theta, const float *__restrict__ dir,
        float *__restrict__ theta_t, __nv_bfloat16 *__restrict__ hi,
        __nv_bfloat16 *__restrict__ lo, const SiteInfo *si, const ChunkInfo *ci, int c0, int c1,
        double *part, const int *counters)
{
    if (counters[2] == 0) return;  // no search continues from the last round
    for (int c = c0 + blockIdx.x; c < c1; c += gridDim.x) {
        const Chunk ch = chunk_at(si, ci, c);
        const SiteState &s = ss[ch.site];
        if (s.status != SITE_SEARCHING || s.trials == 0) continue;
        const float a = (float)s.alpha;
        const int NQ = si[ch.site].NQ, KP = si[ch.site].KP;
        const float4 *t4 = (const float4 *)theta + ch.base4;
        const float4 *d4 = (const float4 *)dir + ch.base4;
        float4 *o4 = (float4 *)theta_t + ch.base4;
        DF acc[2];  // sums of squares: couplings, fields
        for (size_t e = ch.e0 + threadIdx.x; e < ch.e1; e += LB_THREADS) {
            const float4 t = t4[e], dv = d4[e];
            const float4 x = make_float4(fmaf(a, dv.x, t.x), fmaf(a, dv.y, t.y),
                                         fmaf(a, dv.z, t.z), fmaf(a, dv.w, t.w));
            o4[e] = x;
            trial_penalty_split(x, e, ch.base4, NQ, KP, hi, lo, acc[0], acc[1]);
        }
        block_write<2>(acc, part_rec(part, c));
    }
}

// partial g_t . d and ||g_t||^2 (slots 2 and 3; slots 0, 1 hold the penalty)
__global__ void __launch_bounds__(LB_THREADS)
k_ls_dots(const SiteState *ss, const float *__restrict__ g_t, const float *__restrict__ dir,
          const SiteInfo *si, const ChunkInfo *ci, int c0, int c1, double *part)
{
    for (int c = c0 + blockIdx.x; c < c1; c += gridDim.x) {
        const Chunk ch = chunk_at(si, ci, c);
        const SiteState &s = ss[ch.site];
        if (s.status != SITE_SEARCHING) continue;
        const float4 *gt4 = (const float4 *)g_t + ch.base4;
        const float4 *d4 = (const float4 *)dir + ch.base4;
        DF acc[2];
        for (size_t e = ch.e0 + threadIdx.x; e < ch.e1; e += LB_THREADS) {
            const float4 gv = gt4[e], dv = d4[e];
            df_dot4(acc[0], gv, dv);
            df_dot4(acc[1], gv, gv);
        }
        block_write<2>(acc, part_rec(part, c) + 2);
    }
}

__device__ double safe_interp(double lo, double flo, double dlo, double hi, double fhi,
                              double dhi)
{
    // minimiser of the cubic through (lo, flo, dlo) and (hi, fhi, dhi),
    // kept inside the middle 80% of the interval; secant on phi' or
    // bisection otherwise
    const double a = lo, b = hi;
    const double d1 = dlo + dhi - 3.0 * (flo - fhi) / (a - b);
    const double disc = d1 * d1 - dlo * dhi;
    const double L = fmin(a, b), H = fmax(a, b);
    const double mg = 0.1 * (H - L);
    if (disc >= 0.0 && isfinite(disc)) {
        double d2 = sqrt(disc);
        if (b < a) d2 = -d2;
        const double den = dhi - dlo + 2.0 * d2;
        if (den != 0.0) {
            const double t = b - (b - a) * (dhi + d2 - d1) / den;
            if (isfinite(t) && t >= L + mg && t <= H - mg) return t;
        }
    }
    if (dlo < 0.0 && dhi > 0.0) {
        const double t = a - dlo * (b - a) / (dhi - dlo);
        if (isfinite(t) && t >= L + mg && t <= H - mg) return t;
    }
    return 0.5 * (a + b);
}

enum { LS_CONTINUE = 0, LS_ACCEPT = 1, LS_FAIL = 2 };

__global__ void k_ls_decide(SiteState *ss, const double *__restrict__ f_data, const double *part,
                            const SiteInfo *si, int s0, SolveParams p, const int *round_ptr,
                            int *counters)
{
    const int round = *round_ptr;
    const int r = s0 + blockIdx.x;
    SiteState &s = ss[r];
    if (s.status != SITE_SEARCHING) return;
    __shared__ double t4[4];
    if (si[r].nchunks > LB_WARP_SUM_MIN) {
        const int slot[4] = {0, 1, 2, 3};
        double t[4];
        warp_chunk_sums(part, si[r], slot, t);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < 4; ++k) t4[k] = t[k];
    } else if (threadIdx.x < 4) {
        t4[threadIdx.x] = lane_chunk_sum(part, si[r], threadIdx.x);
    }
    __syncwarp();
    if (threadIdx.x != 0) return;
    const double pj = t4[0], ph = t4[1], dgt = t4[2], gn2 = t4[3];
    s.pen_t = p.lambda_h * ph + p.lambda_Jp * pj;
    const double ft = f_data[r] + s.pen_t;
    const double a = s.alpha, f0 = s.f0, dg0 = s.dg0;
    const double eps = p.noise * fmax(1.0, fabs(f0));
    const bool decrease = (ft <= f0 + p.c1 * a * dg0 + eps) || (dgt <= p.c1 * dg0);
    const bool curv = fabs(dgt) <= p.c2 * fabs(dg0);
    int act = LS_CONTINUE;
    s.trials++;
    if (!isfinite(ft) || !isfinite(dgt)) {
        s.a_hi = a;
        s.f_hi = INFINITY;
        s.dg_hi = INFINITY;
        s.phase = 1;
        s.alpha = 0.5 * (s.a_lo + a);
    } else if (decrease && curv) {
        act = LS_ACCEPT;
    } else if (s.phase == 0) {
        if (!decrease || dgt > 0.0) {
            s.a_lo = s.a_prev; s.f_lo = s.f_prev; s.dg_lo = s.dg_prev;
            s.a_hi = a; s.f_hi = ft; s.dg_hi = dgt;
            s.phase = 1;
        } else {
            s.a_prev = a; s.f_prev = ft; s.dg_prev = dgt;
            s.a_lo = a; s.f_lo = ft; s.dg_lo = dgt;
            s.alpha = 4.0 * a;
        }
    } else {
        if (decrease && dgt < 0.0) {
            s.a_lo = a; s.f_lo = ft; s.dg_lo = dgt;
        } else {
            s.a_hi = a; s.f_hi = ft; s.dg_hi = dgt;
        }
    }
    if (act == LS_CONTINUE && s.phase == 1 && isfinite(s.f_hi))
        s.alpha = safe_interp(s.a_lo, s.f_lo, s.dg_lo, s.a_hi, s.f_hi, s.dg_hi);
    if (act == LS_CONTINUE && s.trials >= p.max_ls) act = LS_FAIL;
    if (act == LS_CONTINUE && s.phase == 1 &&
        fabs(s.a_hi - s.a_lo) <= 1e-12 * fmax(s.a_lo, s.a_hi))
        act = LS_FAIL;
    if (act == LS_CONTINUE) {
        atomicAdd(&counters[0], 1);
    } else if (act == LS_ACCEPT) {
        s.commit_round = round;
        s.commit_slot = s.head;
        s.head = (s.head + 1) % p.m;
        if (s.hist < p.m) s.hist++;
        s.f = ft;
        s.gnorm2 = gn2;
        s.iters++;
        if (sqrt(gn2) <= p.gtol) s.status = SITE_CONVERGED;
        else if (s.iters >= p.max_iter) s.status = SITE_FAILED;
        else {
            s.status = SITE_READY;
            atomicAdd(&counters[1], 1);
        }
    } else {
        // a failed search near the optimum is the FP32 noise floor
        s.status = (fabs(ft - f0) <= eps) ? SITE_NOISE : SITE_FAILED;
    }
}

// commit the accepted trial points of this round: s = theta_t - theta,
// y = g_t - g into the ring slot, theta <- theta_t, g <- g_t.  The same pass
// forms what the next direction needs: s_n.g_new and y_n.g_old (slots
// LB_SLOT_SG, LB_SLOT_YG) and, for a site that iterates on, S'y_n and Y'y_n
// over the stored pairs (slots 0..2M-1; the new pair's own entries from
// registers).
template <int M>
__global__ void __launch_bounds__(LB_THREADS, 2)
k_commit(const SiteState *ss, float *__restrict__ theta, float *__restrict__ g,
         const float *__restrict__ theta_t, const float *__restrict__ g_t,
         float *__restrict__ S, float *__restrict__ Y, const SiteInfo *si, const ChunkInfo *ci,
         int c0, int c1, long long vec4, const int *round_ptr, double *part)
{
    const int round = *round_ptr;
    for (int c = c0 + blockIdx.x; c < c1; c += gridDim.x) {
        const Chunk ch = chunk_at(si, ci, c);
        const SiteState &st = ss[ch.site];
        if (st.commit_round != round) continue;
        const int n = st.commit_slot;
        const bool dots = st.status == SITE_READY;
        bool old[M];  // stored pairs other than the new one
#pragma unroll
        for (int j = 0; j < M; ++j) old[j] = dots && j != n && slot_valid(j, st.head, st.hist, M);
        float4 *th4 = (float4 *)theta + ch.base4;
        float4 *g4 = (float4 *)g + ch.base4;
        const float4 *tt4 = (const float4 *)theta_t + ch.base4;
        const float4 *gt4 = (const float4 *)g_t + ch.base4;
        const float4 *S4 = (const float4 *)S + ch.base4;
        const float4 *Y4 = (const float4 *)Y + ch.base4;
        float4 *s4 = (float4 *)S + (size_t)n * vec4 + ch.base4;
        float4 *y4 = (float4 *)Y + (size_t)n * vec4 + ch.base4;
        DF acc[2 * M], sgyg[2];
        for (size_t e = ch.e0 + threadIdx.x; e < ch.e1; e += LB_THREADS) {
            const float4 tn = tt4[e], to = th4[e], gn = gt4[e], go = g4[e];
            float4 sj[M], yj[M];
#pragma unroll
            for (int j = 0; j < M; ++j) {
                sj[j] = old[j] ? S4[(size_t)j * vec4 + e] : f4z();
                yj[j] = old[j] ? Y4[(size_t)j * vec4 + e] : f4z();
            }
            const float4 sv = make_float4(tn.x - to.x, tn.y - to.y, tn.z - to.z, tn.w - to.w);
            const float4 yv = make_float4(gn.x - go.x, gn.y - go.y, gn.z - go.z, gn.w - go.w);
            s4[e] = sv;
            y4[e] = yv;
            th4[e] = tn;
            g4[e] = gn;
            df_dot4(sgyg[0], sv, gn);  // s_n . g_new
            df_dot4(sgyg[1], yv, go);  // y_n . g_old
            if (dots) {
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    const float4 a = (j == n) ? sv : sj[j];
                    const float4 b = (j == n) ? yv : yj[j];
                    df_dot4(acc[j], a, yv);
                    df_dot4(acc[M + j], b, yv);
                }
            }
        }
        if (dots) block_write<2 * M>(acc, part_rec(part, c));
        block_write<2>(sgyg, part_rec(part, c) + LB_SLOT_SG);
    }
}

// resident CTAs of a streaming kernel on this device (at most one per chunk)
template <typename Kern>
int lb_grid(Kern k, int nchunks)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    int slots = 0;
    {
        std::lock_guard<std::mutex> g(mu);
        auto key = std::make_pair((const void *)k, dev);
        auto it = cache.find(key);
        if (it != cache.end()) {
            slots = it->second;
        } else {
            int per_sm = 0, sms = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, LB_THREADS, 0);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            slots = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
            cache[key] = slots;
        }
    }
    return nchunks < slots ? (nchunks > 0 ? nchunks : 1) : slots;
}

// end of a round inside a device-side loop: count the round and continue
// while a site is searching or about to iterate, no tensor-core wait timed
// out and the round cap is not reached
__global__ void k_round_cond(cudaGraphConditionalHandle h, int *counters, int max_rounds)
{
    const int rounds = ++counters[9];
    const bool more =
        (counters[0] + counters[1] > 0) && counters[4] == 0 && rounds < max_rounds;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

}  // namespace

cudaError_t launch_round_cond(cudaGraphConditionalHandle h, int *counters, int max_rounds,
                              cudaStream_t st)
{
    k_round_cond<<<1, 1, 0, st>>>(h, counters, max_rounds);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_lbfgs_init(SiteState *ss, const double *f, const float *g, const LbLayout &L,
                              const SolveParams &p, double *part, cudaStream_t st)
{
    k_init_dots<<<lb_grid(k_init_dots, L.c1 - L.c0), LB_THREADS, 0, st>>>(g, L.si, L.ci, L.c0, L.c1,
                                                                      part);
    k_init_finish<<<L.nsites, 32, 0, st>>>(ss, f, part, L.si, L.s0, p);
    count_launches(2);
    return cudaGetLastError();
}

template <int M>
static void dir_apply_m(SiteState *ss, const float *g, float *dir, const float *S,
                        const float *Y, const float *theta, float *theta_t, __nv_bfloat16 *hi,
                        __nv_bfloat16 *lo, const LbLayout &L, double *part, int *round_ptr,
                        int *counters, cudaStream_t st)
{
    k_dir_solve<M><<<L.nsites, 32, 0, st>>>(ss, part, L.si, L.s0, round_ptr, counters);
    k_dir_apply<M><<<lb_grid(k_dir_apply<M>, L.c1 - L.c0), LB_THREADS, 0, st>>>(
        ss, g, S, Y, dir, theta, theta_t, hi, lo, L.si, L.ci, L.c0, L.c1, L.vec4, part);
}

cudaError_t launch_lbfgs_direction(SiteState *ss, const float *g, float *dir,
                                   const float *S_hist, const float *Y_hist, const float *theta,
                                   float *theta_t, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                                   const LbLayout &L, const SolveParams &p, double *part,
                                   int *round_ptr, int *counters, uint8_t *active,
                                   cudaStream_t st)
{
#define PLM_DIR(MM)                                                                          \
    case MM:                                                                                 \
        dir_apply_m<MM>(ss, g, dir, S_hist, Y_hist, theta, theta_t, hi, lo, L, part,        \
                        round_ptr, counters, st);                                            \
        break;
    switch (p.m) {
        PLM_DIR(1)
        PLM_DIR(2)
        PLM_DIR(3)
        PLM_DIR(4)
        PLM_DIR(5)
        PLM_DIR(6)
        PLM_DIR(7)
        PLM_DIR(8)
    default: return cudaErrorInvalidValue;
    }
#undef PLM_DIR
    k_dir_finish<<<L.nsites, 32, 0, st>>>(ss, part, L.si, L.s0, active);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_lbfgs_trial(SiteState *ss, const float *theta, const float *dir,
                               float *theta_t, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                               const LbLayout &L, double *part, const int *counters,
                               cudaStream_t st)
{
    k_trial<<<lb_grid(k_trial, L.c1 - L.c0), LB_THREADS, 0, st>>>(
        ss, theta, dir, theta_t, hi, lo, L.si, L.ci, L.c0, L.c1, part, counters);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_lbfgs_linesearch(SiteState *ss, const double *f_data, const float *g_t,
                                    const float *dir, const LbLayout &L, const SolveParams &p,
                                    double *part, const int *round_ptr, int *counters,
                                    cudaStream_t st)
{
    k_ls_dots<<<lb_grid(k_ls_dots, L.c1 - L.c0), LB_THREADS, 0, st>>>(ss, g_t, dir, L.si, L.ci,
                                                                        L.c0, L.c1, part);
    k_ls_decide<<<L.nsites, 32, 0, st>>>(ss, f_data, part, L.si, L.s0, p, round_ptr, counters);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_lbfgs_commit(const SiteState *ss, float *theta, float *g,
                                const float *theta_t, const float *g_t, float *S_hist,
                                float *Y_hist, const LbLayout &L, const SolveParams &p,
                                double *part, const int *round_ptr, cudaStream_t st)
{
#define PLM_COMMIT(MM)                                                                       \
    case MM:                                                                                 \
        k_commit<MM><<<lb_grid(k_commit<MM>, L.c1 - L.c0), LB_THREADS, 0, st>>>(         \
            ss, theta, g, theta_t, g_t, S_hist, Y_hist, L.si, L.ci, L.c0, L.c1, L.vec4,     \
            round_ptr, part);                                                                \
        break;
    switch (p.m) {
        PLM_COMMIT(1)
        PLM_COMMIT(2)
        PLM_COMMIT(3)
        PLM_COMMIT(4)
        PLM_COMMIT(5)
        PLM_COMMIT(6)
        PLM_COMMIT(7)
        PLM_COMMIT(8)
    default: return cudaErrorInvalidValue;
    }
#undef PLM_COMMIT
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace plm
