// plm_abi.cu -- the C ABI declared in include/plmdca.h: context and
// workspace management, argument checks, host/device pointer staging, and
// the orchestration of the kernels for each entry point.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/plmdca.h"
#include "plm_internal.cuh"

using namespace plm;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct ProfRecord {
    const char *name;
    cudaEvent_t a, b;
    double bytes;  // algorithmic bytes the bracketed kernels move (0: not counted)
};

constexpr int MAX_LANES = 4;  // lanes of the pipelined solve (counters: 16 ints each)

struct plm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t aux[3] = {nullptr, nullptr, nullptr};  // lanes 1..3 of the pipelined solve
    std::string err;
    std::map<std::string, DevBuf> bufs;
    int *host_counters = nullptr;  // pinned
    double *host_scalars = nullptr;
    bool prof = false;
    std::vector<ProfRecord> prof_records;
    std::vector<cudaEvent_t> event_pool;
};

namespace plm {
void set_error(plm_ctx *c, const char *msg)
{
    if (c) c->err = msg;
}
static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace plm

namespace {

cudaEvent_t take_event(plm_ctx *c)
{
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// brackets the kernels issued in its scope with events when profiling is on
struct ProfScope {
    plm_ctx *c;
    const char *name;
    double bytes;
    cudaEvent_t a = nullptr;
    ProfScope(plm_ctx *c_, const char *n, double bytes_ = 0.0) : c(c_), name(n), bytes(bytes_)
    {
        if (c->prof) {
            a = take_event(c);
            cudaEventRecord(a, c->stream);
        }
    }
    ~ProfScope()
    {
        if (c->prof && a) {
            cudaEvent_t b = take_event(c);
            cudaEventRecord(b, c->stream);
            c->prof_records.push_back({name, a, b, bytes});
        }
    }
};

}  // namespace

namespace plm {
// event hooks for kernels launched outside this file (tensor-core path)
void *prof_start(void *ctx)
{
    plm_ctx *c = (plm_ctx *)ctx;
    cudaEvent_t e = take_event(c);
    cudaEventRecord(e, c->stream);
    return (void *)e;
}

void prof_stop(void *ctx, const char *name, void *start)
{
    plm_ctx *c = (plm_ctx *)ctx;
    cudaEvent_t b = take_event(c);
    cudaEventRecord(b, c->stream);
    c->prof_records.push_back({name, (cudaEvent_t)start, b, 0.0});
}

int identity_threshold(double x, int N)
{
    // smallest integer count T with T / N >= x
    double t = std::ceil(x * (double)N - 1e-9);
    return t < 0 ? 0 : (int)t;
}
}  // namespace plm

namespace {

plm_status fail(plm_ctx *c, plm_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

plm_status cuda_fail(plm_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, e == cudaErrorMemoryAllocation ? PLM_ENOMEM : PLM_ECUDA,
                "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
    } while (0)

// grow-only named workspace buffer
cudaError_t ws(plm_ctx *ctx, const char *name, size_t bytes, void **out)
{
    DevBuf &b = ctx->bufs[name];
    if (bytes == 0) bytes = 256;
    if (b.bytes < bytes) {
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
        cudaError_t e = cudaMalloc(&b.p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        b.bytes = bytes;
    }
    *out = b.p;
    return cudaSuccess;
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// An input array: device pointers are used as they are; host arrays are
// copied into a workspace buffer on the context's stream.
struct Staged {
    void *dev = nullptr;
    void *host = nullptr;  // non-null when results must be copied back
    size_t bytes = 0;
};

cudaError_t stage_in(plm_ctx *ctx, const char *name, const void *p, size_t bytes,
                     const void **out, bool *was_host = nullptr)
{
    if (!p || is_device_ptr(p)) {
        *out = p;
        if (was_host) *was_host = false;
        return cudaSuccess;
    }
    void *d;
    cudaError_t e = ws(ctx, name, bytes, &d);
    if (e) return e;
    e = cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, ctx->stream);
    *out = d;
    if (was_host) *was_host = true;
    return e;
}

cudaError_t stage_out(plm_ctx *ctx, const char *name, void *p, size_t bytes,
                      Staged *s)
{
    s->bytes = bytes;
    if (!p || is_device_ptr(p)) {
        s->dev = p;
        s->host = nullptr;
        return cudaSuccess;
    }
    s->host = p;
    return ws(ctx, name, bytes, &s->dev);
}

cudaError_t copy_back(plm_ctx *ctx, const Staged &s)
{
    if (!s.host) return cudaSuccess;
    return cudaMemcpyAsync(s.host, s.dev, s.bytes, cudaMemcpyDeviceToHost, ctx->stream);
}

__global__ void k_check_msa(const int8_t *msa, size_t n, int *err)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) {
        int s = msa[idx];
        if (s < 0 || s >= Q) atomicOr(err, 1);
    }
}

plm_status check_common(plm_ctx *ctx, int B, int N, int q)
{
    if (!ctx) return PLM_EINVAL;
    if (q != Q) return fail(ctx, PLM_EINVAL, "q must be %d (got %d)", Q, q);
    if (B < 1) return fail(ctx, PLM_EINVAL, "B must be >= 1 (got %d)", B);
    if (N < 2) return fail(ctx, PLM_EINVAL, "N must be >= 2 (got %d)", N);
    if ((long long)N * Q * QP * (long long)N > (1LL << 33))
        return fail(ctx, PLM_EINVAL, "N = %d is too large", N);
    return PLM_OK;
}

// msa validity: a sync point; returns PLM_EINVAL for states outside 0..q-1
plm_status check_msa(plm_ctx *ctx, const int8_t *msa_d, int B, int N)
{
    void *flag;
    CK(ws(ctx, "flag_msa", sizeof(int), &flag));
    CK(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
    size_t n = (size_t)B * N;
    k_check_msa<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(msa_d, n, (int *)flag);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ctx->host_counters + 8, flag, sizeof(int), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->host_counters[8]) return fail(ctx, PLM_EINVAL, "msa has states outside 0..%d", Q - 1);
    return PLM_OK;
}

// ---------------------------------------------------------------------------
// A problem = one or more families solved (or evaluated) together.  Every
// solver vector is an arena holding the padded Theta blocks of the families
// one after another; the sites of family f are sites site0_f .. site0_f+N_f-1.
struct Fam {
    const int8_t *msa = nullptr;  // device
    Dims d;
    size_t off = 0;   // arena offset (floats)
    size_t woff = 0;  // offset in the concatenated weights
    int site0 = 0;
    double beff = 0.0;
};

struct Problem {
    std::vector<Fam> fam;
    size_t total = 0, wtotal = 0;
    int nsites = 0, nchunks = 0;
    int maxB = 0, maxN = 0;
    size_t tc_scratch = 0;
    LbLayout L{};
    std::vector<int> site_chunk0;  // first chunk of each site (host copy of the tables)
    std::vector<TcBatch> tcb;  // the families in launches of at most MAX_FAM
    bool tc_ready = false;
    TcConfig tc_cfg;
    bool tc_tuned = false;
    bool autotune = true;
    // symmetric plmDCA (one family): one L-BFGS problem over the whole arena
    bool symmetric = false;
    int tune_lanes = 1;  // lanes the solve will run (the autotuner times lane-shaped evaluations)
    int lb_sites = 0;              // L-BFGS problems: nsites, or 1 when symmetric
    std::vector<int> lb_len4;      // streamed float4 of each L-BFGS problem
};

void layout_problem(Problem &P)
{
    size_t off = 0, woff = 0;
    int site0 = 0;
    P.tc_scratch = 0;
    for (auto &F : P.fam) {
        F.off = off;
        F.woff = woff;
        F.site0 = site0;
        off += F.d.theta_elems();
        woff += (size_t)F.d.B;
        site0 += F.d.N;
        P.maxB = std::max(P.maxB, F.d.B);
        P.maxN = std::max(P.maxN, F.d.N);
        P.tc_scratch += (tc_family_scratch_bytes(F.d.B, F.d.N) + 255) / 256 * 256;
    }
    P.total = off;
    P.wtotal = woff;
    P.nsites = site0;
}

// site and chunk tables of the batched L-BFGS
plm_status build_lbfgs_tables(plm_ctx *ctx, Problem &P)
{
    std::vector<SiteInfo> si;
    std::vector<ChunkInfo> ci;
    if (P.symmetric) {
        // one problem: every row of the family (padding rows stay zero)
        const Fam &F = P.fam[0];
        const int len4 = (int)(F.d.theta_elems() / 4);
        SiteInfo x;
        x.off4 = (long long)(F.off / 4);
        x.len4 = len4;
        x.KP = F.d.KP;
        x.NQ = F.d.N * Q;
        x.chunk0 = 0;
        x.nchunks = (len4 + LB_CHUNK4 - 1) / LB_CHUNK4;
        x.family = 0;
        x.r = 0;
        for (int c = 0; c < x.nchunks; ++c) {
            ChunkInfo y;
            y.site = 0;
            y.e0 = c * LB_CHUNK4;
            y.e1 = std::min(len4, (c + 1) * LB_CHUNK4);
            ci.push_back(y);
        }
        si.push_back(x);
    }
    for (size_t f = 0; f < P.fam.size() && !P.symmetric; ++f) {
        const Fam &F = P.fam[f];
        // the q state rows of the site; its padding rows (Q..QP-1) stay zero in
        // theta and are never streamed
        const int len4 = Q * F.d.KP / 4;
        const int nch = (len4 + LB_CHUNK4 - 1) / LB_CHUNK4;
        for (int r = 0; r < F.d.N; ++r) {
            SiteInfo x;
            x.off4 = (long long)((F.off + (size_t)r * F.d.site_elems()) / 4);
            x.len4 = len4;
            x.KP = F.d.KP;
            x.NQ = F.d.N * Q;
            x.chunk0 = (int)ci.size();
            x.nchunks = nch;
            x.family = (int)f;
            x.r = r;
            for (int c = 0; c < nch; ++c) {
                ChunkInfo y;
                y.site = (int)si.size();
                y.e0 = c * LB_CHUNK4;
                y.e1 = std::min(len4, (c + 1) * LB_CHUNK4);
                ci.push_back(y);
            }
            si.push_back(x);
        }
    }
    P.site_chunk0.resize(si.size() + 1);
    for (size_t r = 0; r < si.size(); ++r) P.site_chunk0[r] = si[r].chunk0;
    P.lb_sites = (int)si.size();
    P.lb_len4.resize(si.size());
    for (size_t r = 0; r < si.size(); ++r) P.lb_len4[r] = si[r].len4;
    P.site_chunk0[si.size()] = (int)ci.size();
    void *dsi, *dci;
    CK(ws(ctx, "lb_site_info", si.size() * sizeof(SiteInfo), &dsi));
    CK(ws(ctx, "lb_chunk_info", ci.size() * sizeof(ChunkInfo), &dci));
    CK(cudaMemcpyAsync(dsi, si.data(), si.size() * sizeof(SiteInfo), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaMemcpyAsync(dci, ci.data(), ci.size() * sizeof(ChunkInfo), cudaMemcpyHostToDevice,
                       ctx->stream));
    P.nchunks = (int)ci.size();
    P.L.si = (const SiteInfo *)dsi;
    P.L.ci = (const ChunkInfo *)dci;
    P.L.s0 = 0;
    P.L.nsites = P.lb_sites;
    P.L.c0 = 0;
    P.L.c1 = P.nchunks;
    P.L.vec4 = (long long)(P.total / 4);
    return PLM_OK;
}

// tensor-core scratch, transposed MSAs and launch groups (once per problem)
plm_status prepare_tc(plm_ctx *ctx, Problem &P, const float *w)
{
    void *base;
    CK(ws(ctx, "tc_scratch", P.tc_scratch, &base));
    P.tcb.clear();
    size_t at = 0;
    for (size_t f0 = 0; f0 < P.fam.size(); f0 += MAX_FAM) {
        TcBatch b;
        memset(&b, 0, sizeof b);
        std::vector<void *> scr;
        const size_t nf = std::min((size_t)MAX_FAM, P.fam.size() - f0);
        b.nfam = (int)nf;
        for (size_t i = 0; i < nf; ++i) {
            const Fam &F = P.fam[f0 + i];
            FamDesc &D = b.f[i];
            D.msa = F.msa;
            D.w = w + F.woff;
            D.B = F.d.B;
            D.N = F.d.N;
            D.beff = F.beff;
            D.inv_beff = 1.0 / F.beff;
            scr.push_back((char *)base + at);
            at += (tc_family_scratch_bytes(F.d.B, F.d.N) + 255) / 256 * 256;
        }
        CK(launch_tc_prepare(b, scr.data(), ctx->stream));
        P.tcb.push_back(b);
    }
    P.tc_ready = true;
    return PLM_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the tensor-core tile shapes.  For a problem signature (the
// (N, B) of its families) every candidate shape of the logits kernel (sites
// per tile) and of the gradient kernel (columns per tile) is timed with CUDA
// events on the context's stream -- one warm-up launch, then the best of two
// -- and the fastest of each is kept.  The choice is cached per signature for
// the life of the process.  Wave quantisation on 152 SMs is what mostly
// decides it (e.g. 230 vs 276 gradient tiles).
std::mutex g_tune_mutex;
std::map<std::string, TcConfig> g_tune_cache;

std::string problem_signature(const Problem &P)
{
    std::string sig;
    char buf[48];
    for (auto &F : P.fam) {
        snprintf(buf, sizeof buf, "%d:%d;", F.d.N, F.d.B);
        sig += buf;
    }
    return sig;
}

// first sites of the lanes of a one-family pipelined solve: boundaries at
// multiples of lcm(16 or 32, sites per logits group), so that no gradient
// row tile (128 rows = 16/3 sites, or 256 rows) and no logits site group
// straddles two lanes
std::vector<int> lane_bounds(int N, const TcConfig &c, int K)
{
    // gradient row tiles: 6 or 12 sites on one CTA; on CTA pairs 32 sites =
    // 768 padded rows = three 256-row tiles
    const int step = c.gr_pair ? 32 : (c.gr_rows > 128 ? 12 : 6);
    int unit = step;
    while (unit % c.lg_sites) unit += step;
    std::vector<int> b{0};
    for (int k = 1; k < K; ++k) {
        const int h = (int)(((long long)N * k / K + unit / 2) / unit * unit);
        if (h - b.back() >= unit && N - h >= unit) b.push_back(h);
    }
    b.push_back(N);
    return b;
}

plm_status autotune_tc(plm_ctx *ctx, Problem &P, int *tc_err)
{
    const std::string sig = problem_signature(P) + "L" + std::to_string(P.tune_lanes);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(sig);
        if (it != g_tune_cache.end()) {
            P.tc_cfg = it->second;
            P.tc_tuned = true;
            return PLM_OK;
        }
    }
    cudaStream_t st = ctx->stream;
    cudaEvent_t e0 = take_event(ctx), e1 = take_event(ctx);
    // with lanes, a candidate is timed as the lanes launch it: one
    // evaluation per lane, each with that lane's sites active
    const bool laned = P.tune_lanes > 1 && P.fam.size() == 1;
    const int N = P.fam[0].d.N;
    uint8_t *masks = nullptr;
    if (laned) {
        void *m;
        CK(ws(ctx, "tune_masks", (size_t)P.tune_lanes * N, &m));
        masks = (uint8_t *)m;
    }
    const uint8_t *saved_active = P.tcb[0].f[0].active;
    auto time_it = [&](const TcConfig &c, int which, float *best) -> plm_status {
        int nl = 1;
        if (laned) {
            const std::vector<int> b = lane_bounds(N, c, P.tune_lanes);
            nl = (int)b.size() - 1;
            if (nl < P.tune_lanes) {
                // this shape cannot be split into the lanes: not a candidate
                *best = 1e30f;
                return PLM_OK;
            }
            if (which == 2 && !c.gr_pair) {
                // a lane's one-wave gradient grid leaves a fifth of the SMs to
                // the other lanes' L-BFGS passes (about 150 registers a
                // thread, so they cannot share an SM that a gradient CTA
                // holds).  Measured on the family (N = 120, 60-site lanes,
                // 128-row tiles): 120 CTAs a lane 0.029 s per solve, 130
                // 0.029, 140 0.030, 150 0.031-0.032, while timed alone the
                // 150-CTA grid is the fastest.  Grids of several waves hold
                // every SM whatever their width and stay candidates.
                const FamDesc &F = P.tcb[0].f[0];
                const int spt = GR_SITES * c.gr_rows / 128;
                const int nct = (F.KP + c.gr_ncols - 1) / c.gr_ncols;
                for (int k = 0; k < nl; ++k) {
                    const int ctas = (b[k + 1] - b[k] + spt - 1) / spt * nct;
                    if (ctas > num_sms() * 4 / 5 && ctas <= num_sms()) {
                        *best = 1e30f;
                        return PLM_OK;
                    }
                }
            }
            std::vector<uint8_t> h((size_t)nl * N, 0);
            for (int k = 0; k < nl; ++k)
                for (int r = b[k]; r < b[k + 1]; ++r) h[(size_t)k * N + r] = 1;
            CK(cudaMemcpyAsync(masks, h.data(), h.size(), cudaMemcpyHostToDevice, st));
        }
        *best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            CK(cudaEventRecord(e0, st));
            for (int k = 0; k < nl; ++k) {
                if (laned) P.tcb[0].f[0].active = masks + (size_t)k * N;
                for (auto &b : P.tcb)
                    CK(launch_tc_eval(nullptr, b, c, 0.0, 0.0, tc_err, st, which));
            }
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0 && ms < *best) *best = ms;
        }
        P.tcb[0].f[0].active = saved_active;
        return PLM_OK;
    };
    TcConfig best;
    float tbest = 1e30f;
    if (laned && lane_bounds(N, best, P.tune_lanes).size() - 1 < (size_t)P.tune_lanes)
        best.lg_sites = 4;  // a default that splits
    // logits: single-CTA tiles of 4..10 sites, pair tiles of 8, 10 or 12 sites
    const int lg_cand[7][2] = {{4, 0}, {6, 0}, {8, 0}, {10, 0}, {8, 1}, {10, 1}, {12, 1}};
    for (const auto &lc : lg_cand) {
        TcConfig c = best;
        c.lg_sites = lc[0];
        c.lg_pair = lc[1];
        float t;
        plm_status s = time_it(c, 1, &t);
        if (s) return s;
        if (t < tbest) {
            tbest = t;
            best.lg_sites = lc[0];
            best.lg_pair = lc[1];
        }
    }
    tbest = 1e30f;
    // gradient: 128- or 256-row single-CTA tiles, or 256-row tiles on CTA pairs
    // (whose width splits in two halves of a multiple of 16)
    for (int shape : {0, 1, 2})
        for (int cols : {128, 144, 160, 176, 192, 208, 224, 256}) {
            if (shape == 2 && cols % 32) continue;
            TcConfig c = best;
            c.gr_rows = shape == 0 ? 128 : 256;
            c.gr_pair = shape == 2 ? 1 : 0;
            c.gr_ncols = cols;
            float t;
            plm_status s = time_it(c, 2, &t);
            if (s) return s;
            if (t < tbest) {
                tbest = t;
                best.gr_rows = c.gr_rows;
                best.gr_pair = c.gr_pair;
                best.gr_ncols = cols;
            }
        }
    ctx->event_pool.push_back(e0);
    ctx->event_pool.push_back(e1);
    if (getenv("PLMDCA_TC_VERBOSE"))  // the chosen shape, in PLMDCA_TC_TILES form
        fprintf(stderr, "plmdca tiles %s: %d,%d,%d,%d,%d\n", sig.c_str(), best.lg_sites,
                best.gr_ncols, best.gr_rows, best.lg_pair, best.gr_pair);
    P.tc_cfg = best;
    P.tc_tuned = true;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[sig] = best;
    return PLM_OK;
}

// One objective+gradient evaluation of every site of the problem at theta
// (arena).  f_data[site] = -(1/B_eff) sum_b w_b log P (no penalty); G (arena)
// includes 2 lambda theta.
plm_status evaluate(plm_ctx *ctx, plm_precision prec, Problem &P, const float *w,
                    const float *theta, const __nv_bfloat16 *hi, const __nv_bfloat16 *lo,
                    double lambda_h, double lambda_Jp, double *f_data, float *G, int *tc_err,
                    const uint8_t *active = nullptr, cudaStream_t on = nullptr, int which = 3)
{
    cudaStream_t st = on ? on : ctx->stream;
    if (prec == PLM_FP32_EXACT) {
        void *L, *D, *part;
        size_t lmax = 0, pmax = 0;
        for (auto &F : P.fam) {
            lmax = std::max(lmax, (size_t)F.d.B * F.d.R);
            pmax = std::max(pmax, (size_t)softmax_slices(F.d) * F.d.N);
        }
        CK(ws(ctx, "L", lmax * sizeof(float), &L));
        CK(ws(ctx, "D", lmax * sizeof(float), &D));
        CK(ws(ctx, "partial", pmax * sizeof(double), &part));
        for (auto &F : P.fam) {
            const Dims &d = F.d;
            const int slices = softmax_slices(d);
            const float *th = theta + F.off;
            {
                ProfScope ps(ctx, "logits_gather");
                CK(launch_logits_gather(F.msa, th, d, (float *)L,
                                        active ? active + F.site0 : nullptr, st));
            }
            {
                ProfScope ps(ctx, "softmax_resid");
                CK(launch_softmax_resid(F.msa, w + F.woff, F.beff, (float *)L, d, (double *)part,
                                        (float *)D, active ? active + F.site0 : nullptr, st));
                CK(launch_finish_objective((double *)part, slices, d, F.beff, nullptr,
                                           f_data + F.site0, st));
            }
            if (which & 2) {
                ProfScope ps(ctx, "grad_gather");
                CK(launch_grad_gather(F.msa, (float *)D, th, d, lambda_h, lambda_Jp, G + F.off,
                                      active ? active + F.site0 : nullptr, st));
            }
        }
        return PLM_OK;
    }
    if (prec == PLM_SPLIT_BF16) {
        if (!tc_supported())
            return fail(ctx, PLM_ENOTIMPL, "split-bf16 tensor-core path needs an sm_103 GPU");
        if (!P.tc_ready) {
            plm_status s = prepare_tc(ctx, P, w);
            if (s) return s;
        }
        size_t f0 = 0;
        for (auto &b : P.tcb) {
            for (int i = 0; i < b.nfam; ++i) {
                const Fam &F = P.fam[f0 + i];
                FamDesc &D = b.f[i];
                D.th_hi = hi + F.off;
                D.th_lo = lo + F.off;
                D.theta = theta + F.off;
                D.G = G + F.off;
                D.f_data = f_data + F.site0;
                D.active = active ? active + F.site0 : nullptr;
            }
            f0 += b.nfam;
        }
        if (!P.tc_tuned) {
            // PLMDCA_TC_TILES="sites,cols[,rows[,pair[,gradient pair]]]" forces a
            // tile shape (tests, experiments)
            const char *force = getenv("PLMDCA_TC_TILES");
            TcConfig fc;
            if (force &&
                sscanf(force, "%d,%d,%d,%d,%d", &fc.lg_sites, &fc.gr_ncols, &fc.gr_rows, &fc.lg_pair,
                       &fc.gr_pair) >= 2 &&
                tc_config_valid(fc)) {
                P.tc_cfg = fc;
                P.tc_tuned = true;
            } else if (P.autotune) {
                plm_status s = autotune_tc(ctx, P, tc_err);
                if (s) return s;
            } else {
                P.tc_cfg = TcConfig();
                P.tc_tuned = true;
            }
        }
        for (auto &b : P.tcb)
            CK(launch_tc_eval(ctx->prof ? (void *)ctx : nullptr, b, P.tc_cfg, lambda_h, lambda_Jp,
                              tc_err, st, which));
        return PLM_OK;
    }
    return fail(ctx, PLM_ENOTIMPL, "precision mode %d is not built", (int)prec);
}

struct SolveOut {
    float *h, *J;        // device (possibly staged)
    plm_report *report;  // host, may be NULL
};

// Steps 1-3 for every family of the problem; outputs unpacked per family.
plm_status solve_core(plm_ctx *ctx, Problem &P, const plm_opts &o, std::vector<SolveOut> &out,
                      std::vector<plm_report> &reps)
{
    auto t_start = std::chrono::steady_clock::now();
    cudaStream_t st = ctx->stream;
    layout_problem(P);
    const size_t nf = P.fam.size();

    // step 2: reweighting, per family
    void *scratch, *w, *beff_d, *flag;
    CK(ws(ctx, "rw_scratch", reweight_scratch_bytes(P.maxB, P.maxN), &scratch));
    CK(ws(ctx, "w", P.wtotal * sizeof(float), &w));
    CK(ws(ctx, "beff", nf * sizeof(double), &beff_d));
    CK(ws(ctx, "flag_rw", sizeof(int), &flag));
    CK(cudaMemsetAsync(flag, 0, sizeof(int), st));
    {
        ProfScope ps(ctx, "reweight");
        for (size_t f = 0; f < nf; ++f) {
            const Fam &F = P.fam[f];
            CK(launch_reweight(F.msa, F.d.B, F.d.N, identity_threshold(o.x, F.d.N), nullptr,
                               (float *)w + F.woff, (double *)beff_d + f, scratch, (int *)flag,
                               st));
        }
    }
    std::vector<double> beffs(nf);
    CK(cudaMemcpyAsync(ctx->host_counters + 9, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(beffs.data(), beff_d, nf * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (ctx->host_counters[9]) return fail(ctx, PLM_EINVAL, "msa has states outside 0..%d", Q - 1);
    for (size_t f = 0; f < nf; ++f) P.fam[f].beff = beffs[f];

    plm_status s = build_lbfgs_tables(ctx, P);
    if (s) return s;
    P.tc_ready = false;

    // workspace of the solver
    const size_t tb = P.total * sizeof(float);
    void *theta, *theta_t, *g, *g_t, *dir, *Sh, *Yh, *sst, *fdat, *cnt, *part;
    void *hi = nullptr, *lo = nullptr;
    CK(ws(ctx, "theta", tb, &theta));
    CK(ws(ctx, "theta_t", tb, &theta_t));
    CK(ws(ctx, "g", tb, &g));
    CK(ws(ctx, "G", tb, &g_t));
    CK(ws(ctx, "dir", tb, &dir));
    CK(ws(ctx, "S_hist", tb * o.lbfgs_m, &Sh));
    CK(ws(ctx, "Y_hist", tb * o.lbfgs_m, &Yh));
    CK(ws(ctx, "site_state", (size_t)P.lb_sites * sizeof(SiteState), &sst));
    // per-site data terms, and (symmetric) their sum in the last slot
    CK(ws(ctx, "fdata", (size_t)(P.nsites + 1) * sizeof(double), &fdat));
    double *f_lb = (double *)fdat + (P.symmetric ? P.nsites : 0);  // what the line search reads
    CK(ws(ctx, "counters", 16 * MAX_LANES * sizeof(int), &cnt));  // 16 per lane (see below)
    CK(ws(ctx, "lb_part", (size_t)P.nchunks * LB_PART * sizeof(double), &part));
    void *active;
    CK(ws(ctx, "active", MAX_LANES * (size_t)P.nsites, &active));  // one flag array per lane
    if (o.prec == PLM_SPLIT_BF16) {
        CK(ws(ctx, "theta_hi", P.total * 2, &hi));
        CK(ws(ctx, "theta_lo", P.total * 2, &lo));
    }
    SolveParams p;
    p.lambda_h = o.lambda_h;
    p.lambda_Jp = 0.5 * o.lambda_J;  // step 1 of the rundown
    p.gtol = o.gtol;
    p.c1 = 1e-4;
    p.c2 = 0.9;
    p.noise = 1e-6;
    p.m = o.lbfgs_m;
    p.max_iter = o.max_iter;
    p.max_ls = o.max_ls;

    // origin start (Sec. 6)
    CK(cudaMemsetAsync(theta, 0, tb, st));
    CK(cudaMemsetAsync(theta_t, 0, tb, st));
    CK(cudaMemsetAsync(dir, 0, tb, st));
    if (hi) {
        CK(cudaMemsetAsync(hi, 0, P.total * 2, st));
        CK(cudaMemsetAsync(lo, 0, P.total * 2, st));
    }
    int evals = 0;
    int *tc_err = (int *)cnt + 4;  // tensor-core timeout word, read back with the counters
    const bool use_graph = o.use_graph && st != nullptr && !ctx->prof;
    int K = 2;  // lanes of a one-family pipelined solve (PLMDCA_LANES overrides: 1..4)
    if (const char *e = getenv("PLMDCA_LANES")) K = std::max(1, std::min(MAX_LANES, atoi(e)));
    const bool pipelined = use_graph && o.prec == PLM_SPLIT_BF16 && !P.symmetric;
    P.tune_lanes = (pipelined && nf == 1) ? K : 1;
    CK(cudaMemsetAsync(cnt, 0, 16 * MAX_LANES * sizeof(int), st));
    CK(cudaMemsetAsync(active, 0, MAX_LANES * (size_t)P.nsites, st));
    s = evaluate(ctx, o.prec, P, (const float *)w, (const float *)theta,
                 (const __nv_bfloat16 *)hi, (const __nv_bfloat16 *)lo, p.lambda_h, p.lambda_Jp,
                 (double *)fdat, (float *)g, tc_err);
    if (s) return s;
    if (P.symmetric) {
        // the symmetric problem's gradient and objective (data part)
        CK(launch_sym_project((float *)g, P.fam[0].d, st));
        CK(launch_sum_sites((const double *)fdat, P.nsites, f_lb, st));
    }
    evals++;
    CK(launch_lbfgs_init((SiteState *)sst, f_lb, (const float *)g, P.L, p, (double *)part, st));

    // ---- the rounds.  One round advances every live site of a lane by one
    // evaluation: sites whose last trial was accepted (READY) first form
    // their next direction and first trial point, searching sites take their
    // next trial point, all trial points of the lane are evaluated together
    // and each site's line search decides.  A site never waits for the line
    // searches of other sites, and its iterates do not depend on them (each
    // site's objective involves only its own row block), so a lane needs
    // about max over its sites of that site's evaluations rounds.
    //
    // On the tensor-core path the sites are split into lanes (two by
    // default; PLMDCA_LANES=1..4 for measurements): for one family at
    // boundaries shared by the logits site groups and the 128-row gradient
    // tiles, for a batch at family boundaries.  Each lane has its own
    // counters, round number and active flags, its own stream and CUDA
    // graph, and starts its round at a different phase (lane k at phase
    // k mod 3: direction, evaluation, decision), so one lane's tensor-core
    // evaluation runs while another streams its L-BFGS vectors.  Measured
    // on the family workload: 1 lane 0.035 s, 2 lanes 0.030 s, 3 or 4
    // lanes 0.032 s.  Every other case runs one lane.
    struct Lane {
        LbLayout L;
        int *cnt;          // 16 ints: [0] searching, [1] ready, [2] continuing, [4] tc error, [8] round, [9] rounds
        uint8_t *active;   // evaluation flags (nsites; only this lane's sites set)
        int *hc;           // pinned host copy of cnt[0..4]
        cudaStream_t st;
        cudaGraphExec_t graph = nullptr;
        int offset = 0;  // phase the lane's round starts at: 0 direction, 1 evaluation, 2 decision
        bool done = false;
        int rounds = 0;
    };
    // lane boundaries (sites): [0, b_1, ..., lb_sites]
    std::vector<int> bounds{0, P.lb_sites};
    if (pipelined && P.tc_tuned) {
        std::vector<int> b{0};
        if (nf == 1) {
            b = lane_bounds(P.fam[0].d.N, P.tc_cfg, K);
            b.pop_back();
        } else {
            // whole families per lane (no tile straddles a family), boundaries
            // that best balance the evaluation work B_f N_f^2
            std::vector<double> cum(nf + 1, 0.0);
            for (size_t f = 0; f < nf; ++f)
                cum[f + 1] = cum[f] + (double)P.fam[f].d.B * P.fam[f].d.N * P.fam[f].d.N;
            size_t prev = 0;
            for (int k = 1; k < K; ++k) {
                size_t best = 0;
                double bd = 1e300;
                for (size_t f = prev + 1; f < nf; ++f) {
                    const double d = std::fabs(cum[f] - cum[nf] * k / K);
                    if (d < bd) {
                        bd = d;
                        best = f;
                    }
                }
                if (best > prev) {
                    b.push_back(P.fam[best].site0);
                    prev = best;
                }
            }
        }
        b.push_back(P.lb_sites);
        bounds = b;
    }
    const int nlanes = (int)bounds.size() - 1;
    std::vector<Lane> lanes(nlanes);
    for (int k = 1; k < nlanes; ++k)
        if (!ctx->aux[k - 1]) {
            cudaError_t e = cudaStreamCreateWithFlags(&ctx->aux[k - 1], cudaStreamNonBlocking);
            if (e) return cuda_fail(ctx, e, "cudaStreamCreateWithFlags");
        }
    for (int k = 0; k < nlanes; ++k) {
        Lane &ln = lanes[k];
        ln.L = P.L;
        ln.L.s0 = bounds[k];
        ln.L.nsites = bounds[k + 1] - bounds[k];
        ln.L.c0 = P.site_chunk0[bounds[k]];
        ln.L.c1 = P.site_chunk0[bounds[k + 1]];
        ln.cnt = (int *)cnt + 16 * k;
        ln.active = (uint8_t *)active + (size_t)P.nsites * k;
        ln.hc = ctx->host_counters + 16 * k;
        ln.st = k == 0 ? st : ctx->aux[k - 1];
        ln.offset = k % 3;  // the lane's round starts at this phase
    }

    // algorithmic bytes of the passes of one round, from the site states at
    // its start and after it (profiling only, one lane: each pass streams
    // the elements of the sites it acts on, once per vector it reads or
    // writes)
    struct RoundBytes {
        double dir = 0, trial = 0, ls = 0;
    } rb;
    std::vector<SiteState> snap;
    std::vector<double> site_bytes;  // 4 x streamed elements of each site
    if (ctx->prof) {
        snap.resize(P.lb_sites);
        for (int r = 0; r < P.lb_sites; ++r) site_bytes.push_back(16.0 * P.lb_len4[r]);
    }
    const double split_b = o.prec == PLM_SPLIT_BF16 ? 1.0 : 0.0;  // hi + lo: 2 + 2 B an element
    auto count_round = [&]() -> plm_status {
        CK(cudaMemcpyAsync(snap.data(), sst, snap.size() * sizeof(SiteState),
                           cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        rb = RoundBytes{};
        for (int r = 0; r < P.lb_sites; ++r) {
            const SiteState &x = snap[r];
            const double e = site_bytes[r];
            if (x.status == SITE_READY) {
                // g, S_j, Y_j, theta in; d, theta_t (+ hi, lo) out
                rb.dir += (2.0 * x.hist + 4.0 + split_b) * e;
                rb.ls += 2.0 * e;  // g_t, d in
            } else if (x.status == SITE_SEARCHING) {
                rb.trial += (3.0 + split_b) * e;  // theta, d in; theta_t (+ hi, lo) out
                rb.ls += 2.0 * e;
            }
        }
        return PLM_OK;
    };
    int commit_rec = -1;  // profile record of this round's commit pass
    // the three phases of a round
    auto phase_dir = [&](Lane &ln) -> plm_status {
        if (ctx->prof) {
            plm_status s2 = count_round();
            if (s2) return s2;
        }
        {
            // also starts the round (counter, counts) and sets the active flags
            ProfScope ps(ctx, "lbfgs_direction", rb.dir);
            CK(launch_lbfgs_direction((SiteState *)sst, (const float *)g, (float *)dir,
                                      (const float *)Sh, (const float *)Yh, (const float *)theta,
                                      (float *)theta_t, (__nv_bfloat16 *)hi, (__nv_bfloat16 *)lo,
                                      ln.L, p, (double *)part, ln.cnt + 8, ln.cnt, ln.active,
                                      ln.st));
        }
        {
            ProfScope ps(ctx, "lbfgs_trial", rb.trial);
            CK(launch_lbfgs_trial((SiteState *)sst, (const float *)theta, (const float *)dir,
                                  (float *)theta_t, (__nv_bfloat16 *)hi, (__nv_bfloat16 *)lo,
                                  ln.L, (double *)part, (const int *)ln.cnt, ln.st));
        }
        return PLM_OK;
    };
    auto phase_eval = [&](Lane &ln) -> plm_status {
        plm_status s2 = evaluate(ctx, o.prec, P, (const float *)w, (const float *)theta_t,
                                 (const __nv_bfloat16 *)hi, (const __nv_bfloat16 *)lo,
                                 p.lambda_h, p.lambda_Jp, (double *)fdat, (float *)g_t,
                                 ln.cnt + 4, P.symmetric ? nullptr : ln.active, ln.st);
        if (s2) return s2;
        if (P.symmetric) {
            CK(launch_sym_project((float *)g_t, P.fam[0].d, ln.st));
            CK(launch_sum_sites((const double *)fdat, P.nsites, f_lb, ln.st));
        }
        return PLM_OK;
    };
    auto phase_post = [&](Lane &ln, bool copy_counts) -> plm_status {
        {
            ProfScope ps(ctx, "lbfgs_linesearch", rb.ls);
            CK(launch_lbfgs_linesearch((SiteState *)sst, f_lb, (const float *)g_t,
                                       (const float *)dir, ln.L, p, (double *)part, ln.cnt + 8,
                                       ln.cnt, ln.st));
        }
        {
            ProfScope ps(ctx, "lbfgs_commit");
            CK(launch_lbfgs_commit((const SiteState *)sst, (float *)theta, (float *)g,
                                   (const float *)theta_t, (const float *)g_t, (float *)Sh,
                                   (float *)Yh, ln.L, p, (double *)part, ln.cnt + 8, ln.st));
        }
        if (ctx->prof) commit_rec = (int)ctx->prof_records.size() - 1;
        if (copy_counts)
            CK(cudaMemcpyAsync(ln.hc, ln.cnt, 5 * sizeof(int), cudaMemcpyDeviceToHost, ln.st));
        return PLM_OK;
    };
    // every site stops within max_iter iterations of at most max_ls trials
    const long long max_rounds = (long long)o.max_iter * o.max_ls + 1;
    const int max_rounds_i = (int)std::min<long long>(max_rounds, 1 << 30);
    // one round; inside a device loop it ends by setting the loop condition
    // instead of copying the counts to the host
    auto round_step = [&](Lane &ln, cudaGraphConditionalHandle cond, bool in_loop) -> plm_status {
        plm_status s2;
        for (int ph = 0; ph < 3; ++ph) {
            const int which = (ln.offset + ph) % 3;
            if (which == 0) s2 = phase_dir(ln);
            else if (which == 1) s2 = phase_eval(ln);
            else {
                s2 = phase_post(ln, !in_loop);
                // the loop condition right after the decisions it reads
                if (!s2 && in_loop) CK(launch_round_cond(cond, ln.cnt, max_rounds_i, ln.st));
            }
            if (s2) return s2;
        }
        return PLM_OK;
    };
    struct GraphGuard {
        std::vector<Lane> *l;
        ~GraphGuard()
        {
            for (auto &ln : *l)
                if (ln.graph) cudaGraphExecDestroy(ln.graph);
        }
    } guard{&lanes};
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> joins(nlanes, nullptr);
    struct EventGuard {
        cudaEvent_t *a;
        std::vector<cudaEvent_t> *b;
        ~EventGuard()
        {
            if (*a) cudaEventDestroy(*a);
            for (auto e : *b)
                if (e) cudaEventDestroy(e);
        }
    } eguard{&fork, &joins};
    if (nlanes > 1) {
        // the other lanes start after everything queued so far on the caller's stream
        CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        CK(cudaEventRecord(fork, st));
        for (int k = 1; k < nlanes; ++k) {
            CK(cudaStreamWaitEvent(lanes[k].st, fork, 0));
            // the phases of the first round before the lane's starting phase
            for (int ph = 0; ph < lanes[k].offset; ++ph) {
                s = ph == 0 ? phase_dir(lanes[k]) : phase_eval(lanes[k]);
                if (s) return s;
            }
        }
    }
    if (use_graph) {
        // each lane's rounds run as one CUDA graph: a while node whose body
        // is the round, the loop condition set on the device at the end of
        // each round, so no round waits for the host
        int body_kernels = 0;
        for (auto &ln : lanes) {
            cudaGraph_t top;
            CK(cudaGraphCreate(&top, 0));
            struct TopGuard {
                cudaGraph_t g;
                ~TopGuard() { cudaGraphDestroy(g); }
            } tg{top};
            cudaGraphConditionalHandle cond;
            CK(cudaGraphConditionalHandleCreate(&cond, top, 1, cudaGraphCondAssignDefault));
            cudaGraphNodeParams np = {};
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = cond;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t node;
            CK(cudaGraphAddNode(&node, top, nullptr, nullptr, 0, &np));
            cudaGraph_t body = np.conditional.phGraph_out[0];
            const long long before = g_launches.load();
            CK(cudaStreamBeginCaptureToGraph(ln.st, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
            plm_status s2 = round_step(ln, cond, true);
            cudaGraph_t captured;
            cudaError_t e = cudaStreamEndCapture(ln.st, &captured);
            // capture records the launches without running them: counted per round below
            body_kernels = (int)(g_launches.load() - before);
            count_launches(-body_kernels);
            if (s2) return s2;
            if (e) return cuda_fail(ctx, e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&ln.graph, top, 0);
            if (e) return cuda_fail(ctx, e, "cudaGraphInstantiate");
        }
        for (auto &ln : lanes) CK(cudaGraphLaunch(ln.graph, ln.st));
        for (auto &ln : lanes) {
            CK(cudaMemcpyAsync(ln.hc, ln.cnt, 10 * sizeof(int), cudaMemcpyDeviceToHost, ln.st));
            CK(cudaStreamSynchronize(ln.st));
            ln.rounds = ln.hc[9];
            count_launches(body_kernels * ln.rounds);
            if (ln.hc[4])
                return fail(ctx, PLM_ETIMEOUT, "tensor-core pipeline wait timed out (code 0x%x)",
                            ln.hc[4]);
        }
    } else {
        for (long long rd = 0; rd < max_rounds; ++rd) {
            for (auto &ln : lanes) {
                if (ln.done) continue;
                s = round_step(ln, 0, false);
                if (s) return s;
                ln.rounds++;
            }
            for (auto &ln : lanes) CK(cudaStreamSynchronize(ln.st));
            if (ctx->prof && commit_rec >= 0) {
                // committed sites: theta_t, theta, g_t, g in; s, y, theta, g out; and
                // the stored pairs other than the new one for a site that iterates on
                CK(cudaMemcpyAsync(snap.data(), sst, snap.size() * sizeof(SiteState),
                                   cudaMemcpyDeviceToHost, st));
                int rd_now = 0;
                CK(cudaMemcpyAsync(&rd_now, lanes[0].cnt + 8, sizeof(int),
                                   cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                double cb = 0.0;
                for (int r = 0; r < P.lb_sites; ++r)
                    if (snap[r].commit_round == rd_now)
                        cb += (8.0 + (snap[r].status == SITE_READY ? 2.0 * (snap[r].hist - 1)
                                                                    : 0.0)) *
                              site_bytes[r];
                ctx->prof_records[commit_rec].bytes = cb;
            }
            bool all_done = true;
            for (auto &ln : lanes) {
                if (ln.hc[4])
                    return fail(ctx, PLM_ETIMEOUT,
                                "tensor-core pipeline wait timed out (code 0x%x)", ln.hc[4]);
                // no site searching or about to iterate
                if (!ln.done && ln.hc[0] == 0 && ln.hc[1] == 0) ln.done = true;
                all_done = all_done && ln.done;
            }
            if (all_done) break;
        }
    }
    for (auto &ln : lanes) evals = std::max(evals, 1 + ln.rounds);
    for (int k = 1; k < nlanes; ++k) {
        // the caller's stream resumes after the other lanes
        CK(cudaEventCreateWithFlags(&joins[k], cudaEventDisableTiming));
        CK(cudaEventRecord(joins[k], lanes[k].st));
        CK(cudaStreamWaitEvent(st, joins[k], 0));
    }

    for (size_t f = 0; f < nf; ++f)
        CK(launch_unpack_theta((const float *)theta + P.fam[f].off, P.fam[f].d, out[f].h,
                               out[f].J, st));
    std::vector<SiteState> host(P.lb_sites);
    CK(cudaMemcpyAsync(host.data(), sst, (size_t)P.lb_sites * sizeof(SiteState),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double secs =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    reps.assign(nf, plm_report{});
    for (size_t f = 0; f < nf; ++f) {
        plm_report &rep = reps[f];
        memset(&rep, 0, sizeof rep);
        rep.evals = evals;
        rep.beff = P.fam[f].beff;
        rep.seconds = secs;
        if (P.symmetric) {
            // one problem: every site shares its outcome
            const SiteState &x = host[0];
            rep.iters = x.iters;
            rep.f_total = x.f;
            rep.gnorm_max = std::sqrt(x.gnorm2);
            const int N = P.fam[f].d.N;
            if (x.status == SITE_CONVERGED) rep.n_converged = N;
            else if (x.status == SITE_NOISE) rep.n_noise = N;
            else rep.n_failed = N;
            continue;
        }
        for (int r = 0; r < P.fam[f].d.N; ++r) {
            const SiteState &x = host[P.fam[f].site0 + r];
            rep.iters = std::max(rep.iters, x.iters);
            rep.f_total += x.f;
            rep.gnorm_max = std::max(rep.gnorm_max, std::sqrt(x.gnorm2));
            if (x.status == SITE_CONVERGED) rep.n_converged++;
            else if (x.status == SITE_NOISE) rep.n_noise++;
            else rep.n_failed++;
        }
    }
    return PLM_OK;
}

plm_status check_opts(plm_ctx *ctx, const plm_opts &o)
{
    if (!(o.x >= 0.0 && o.x <= 1.0)) return fail(ctx, PLM_EINVAL, "x must lie in [0, 1]");
    if (o.lambda_h < 0 || o.lambda_J < 0) return fail(ctx, PLM_EINVAL, "negative lambda");
    if (!(o.lambda_h > 0 && o.lambda_J > 0))
        return fail(ctx, PLM_EINVAL, "lambda_h and lambda_J must be > 0 (the l2 term makes "
                                     "each site problem strongly convex)");
    if (o.lbfgs_m < 1 || o.lbfgs_m > MAX_M)
        return fail(ctx, PLM_EINVAL, "lbfgs_m must be 1..%d", MAX_M);
    if (o.max_ls < 1) return fail(ctx, PLM_EINVAL, "max_ls must be >= 1");
    if (!(o.gtol >= 0)) return fail(ctx, PLM_EINVAL, "gtol must be >= 0");
    if (o.prec != PLM_FP32_EXACT && o.prec != PLM_SPLIT_BF16)
        return fail(ctx, PLM_ENOTIMPL, "precision mode %d is not built", (int)o.prec);
    return PLM_OK;
}

}  // namespace

extern "C" {

void plm_default_opts(plm_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->x = 0.8;
    o->lambda_h = 0.01;
    o->lambda_J = 0.01;
    o->gtol = 1e-4;
    o->lbfgs_m = 5;
    o->max_iter = 1000;
    o->max_ls = 20;
    o->prec = PLM_SPLIT_BF16;
    o->use_graph = 1;
    o->autotune = 1;
}

plm_status plm_create(plm_ctx **out, int device, void *cuda_stream)
{
    if (!out) return PLM_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return PLM_ECUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return PLM_ECUDA;
    plm_ctx *c = new plm_ctx;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaMallocHost(&c->host_counters, 64 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&c->host_scalars, 64 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return PLM_ENOMEM;
    }
    *out = c;
    return PLM_OK;
}

plm_status plm_destroy(plm_ctx *c)
{
    if (!c) return PLM_EINVAL;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    for (auto &a : c->aux)
        if (a) {
            cudaStreamSynchronize(a);
            cudaStreamDestroy(a);
        }
    for (auto &kv : c->bufs)
        if (kv.second.p) cudaFree(kv.second.p);
    if (c->host_counters) cudaFreeHost(c->host_counters);
    if (c->host_scalars) cudaFreeHost(c->host_scalars);
    for (auto &r : c->prof_records) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    delete c;
    return PLM_OK;
}

long long plm_kernel_launches(void) { return plm::g_launches.load(); }

plm_status plm_selftest_wait(plm_ctx *ctx, int *code_out)
{
    using namespace plm;
    if (!ctx) return PLM_EINVAL;
    if (code_out) *code_out = 0;
    cudaSetDevice(ctx->device);
    void *flag;
    CK(ws(ctx, "flag_selftest", sizeof(int), &flag));
    CK(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
    CK(launch_wait_selftest((int *)flag, ctx->stream));
    CK(cudaMemcpyAsync(ctx->host_counters + 11, flag, sizeof(int), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int code = ctx->host_counters[11];
    if (code_out) *code_out = code;
    if (code)
        return fail(ctx, PLM_ETIMEOUT, "device wait gave up as designed (code 0x%x)", code);
    return fail(ctx, PLM_ECUDA, "the bounded wait did not report its timeout");
}

plm_status plm_profile(plm_ctx *c, int enable)
{
    if (!c) return PLM_EINVAL;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto &r : c->prof_records) {
        c->event_pool.push_back(r.a);
        c->event_pool.push_back(r.b);
    }
    c->prof_records.clear();
    c->prof = enable != 0;
    return PLM_OK;
}

int plm_profile_report(plm_ctx *c, char *buf, int len)
{
    if (!c) return -1;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    struct Agg {
        long long n = 0;
        double ms = 0.0, bytes = 0.0;
    };
    std::map<std::string, Agg> agg;
    std::vector<std::string> order;
    for (auto &r : c->prof_records) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto it = agg.find(r.name);
        if (it == agg.end()) order.push_back(r.name);
        Agg &x = agg[r.name];
        x.n++;
        x.ms += ms;
        x.bytes += r.bytes;
    }
    std::string out;
    char line[256];
    for (auto &n : order) {
        snprintf(line, sizeof line, "%s %lld %.6f %.0f\n", n.c_str(), agg[n].n, agg[n].ms,
                 agg[n].bytes);
        out += line;
    }
    if (buf && len > 0) {
        size_t k = out.size() < (size_t)(len - 1) ? out.size() : (size_t)(len - 1);
        memcpy(buf, out.data(), k);
        buf[k] = 0;
    }
    return (int)out.size() + 1;
}

const char *plm_last_error(plm_ctx *c)
{
    return c ? c->err.c_str() : "null context";
}

plm_status msa_reweight(plm_ctx *ctx, const int8_t *msa, int B, int N, int q,
                        double x, int32_t *m_out, float *w_out, double *beff_out)
{
    if (!ctx) return PLM_EINVAL;
    if (q != Q) return fail(ctx, PLM_EINVAL, "q must be %d (got %d)", Q, q);
    if (B < 1 || N < 1) return fail(ctx, PLM_EINVAL, "B and N must be >= 1");
    if (!msa) return fail(ctx, PLM_EINVAL, "msa is NULL");
    if (!(x >= 0.0 && x <= 1.0)) return fail(ctx, PLM_EINVAL, "x must lie in [0, 1]");
    CK(cudaSetDevice(ctx->device));
    const void *msa_d;
    CK(stage_in(ctx, "in_msa", msa, (size_t)B * N, &msa_d));
    Staged m_s, w_s;
    CK(stage_out(ctx, "out_m", m_out, (size_t)B * sizeof(int32_t), &m_s));
    CK(stage_out(ctx, "out_w", w_out, (size_t)B * sizeof(float), &w_s));
    void *scratch, *beff_d, *flag;
    CK(ws(ctx, "rw_scratch", reweight_scratch_bytes(B, N), &scratch));
    CK(ws(ctx, "beff", sizeof(double), &beff_d));
    CK(ws(ctx, "flag_rw", sizeof(int), &flag));
    CK(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
    CK(launch_reweight((const int8_t *)msa_d, B, N, identity_threshold(x, N),
                       (int32_t *)m_s.dev, (float *)w_s.dev, (double *)beff_d, scratch,
                       (int *)flag, ctx->stream));
    CK(copy_back(ctx, m_s));
    CK(copy_back(ctx, w_s));
    CK(cudaMemcpyAsync(ctx->host_scalars, beff_d, sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->host_counters + 9, flag, sizeof(int), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->host_counters[9]) return fail(ctx, PLM_EINVAL, "msa has states outside 0..%d", Q - 1);
    if (beff_out) *beff_out = ctx->host_scalars[0];
    return PLM_OK;
}

plm_status plm_site_objective_grad(plm_ctx *ctx, const int8_t *msa,
                                   const float *w, double beff, int B, int N,
                                   int q, const float *h, const float *J,
                                   double lambda_h, double lambda_J,
                                   plm_precision prec, double *f_out,
                                   float *gh, float *gJ)
{
    plm_status s = check_common(ctx, B, N, q);
    if (s) return s;
    if (!msa || !w || !h || !J) return fail(ctx, PLM_EINVAL, "null input array");
    if (!(beff > 0.0)) return fail(ctx, PLM_EINVAL, "beff must be > 0");
    if (lambda_h < 0 || lambda_J < 0) return fail(ctx, PLM_EINVAL, "negative lambda");
    if ((gh == nullptr) != (gJ == nullptr))
        return fail(ctx, PLM_EINVAL, "gh and gJ must both be given or both be NULL");
    const int which = gh ? 3 : 1;  // no gradient asked for: the logits pass only
    CK(cudaSetDevice(ctx->device));
    const Dims d = make_dims(B, N);
    const size_t NQ = (size_t)N * Q;
    const void *msa_d, *w_d, *h_d, *J_d;
    CK(stage_in(ctx, "in_msa", msa, (size_t)B * N, &msa_d));
    s = check_msa(ctx, (const int8_t *)msa_d, B, N);
    if (s) return s;
    CK(stage_in(ctx, "in_w", w, (size_t)B * sizeof(float), &w_d));
    CK(stage_in(ctx, "in_h", h, NQ * sizeof(float), &h_d));
    CK(stage_in(ctx, "in_J", J, NQ * NQ * sizeof(float), &J_d));
    Staged f_s, gh_s, gJ_s;
    CK(stage_out(ctx, "out_f", f_out, (size_t)N * sizeof(double), &f_s));
    CK(stage_out(ctx, "out_gh", gh, NQ * sizeof(float), &gh_s));
    CK(stage_out(ctx, "out_gJ", gJ, NQ * NQ * sizeof(float), &gJ_s));
    Problem P;
    Fam F;
    F.msa = (const int8_t *)msa_d;
    F.d = d;
    F.beff = beff;
    P.fam.push_back(F);
    layout_problem(P);
    void *theta, *G, *pen, *fdat, *hi = nullptr, *lo = nullptr;
    CK(ws(ctx, "theta", d.theta_elems() * sizeof(float), &theta));
    CK(ws(ctx, "G", d.theta_elems() * sizeof(float), &G));
    CK(ws(ctx, "pen", (size_t)N * sizeof(double), &pen));
    CK(ws(ctx, "fdata", (size_t)N * sizeof(double), &fdat));
    const double lJp = 0.5 * lambda_J;  // step 1 of the rundown
    CK(launch_pack_theta((const float *)h_d, (const float *)J_d, d, (float *)theta, ctx->stream));
    CK(launch_penalty((const float *)theta, d, lambda_h, lJp, (double *)pen, ctx->stream));
    if (prec == PLM_SPLIT_BF16) {
        CK(ws(ctx, "theta_hi", d.theta_elems() * 2, &hi));
        CK(ws(ctx, "theta_lo", d.theta_elems() * 2, &lo));
        CK(launch_split_theta((const float *)theta, d.theta_elems(), (__nv_bfloat16 *)hi,
                              (__nv_bfloat16 *)lo, ctx->stream));
    }
    void *tcflag;
    CK(ws(ctx, "flag_tc", sizeof(int), &tcflag));
    CK(cudaMemsetAsync(tcflag, 0, sizeof(int), ctx->stream));
    s = evaluate(ctx, prec, P, (const float *)w_d, (const float *)theta,
                 (const __nv_bfloat16 *)hi, (const __nv_bfloat16 *)lo, lambda_h, lJp,
                 (double *)fdat, (float *)G, (int *)tcflag, nullptr, nullptr, which);
    if (s) return s;
    // f = data + penalty (the finishing kernel with one "slice" and B_eff = -1
    // computes -(-fdata) + pen)
    void *fsum;
    CK(ws(ctx, "fsum", (size_t)N * sizeof(double), &fsum));
    CK(launch_finish_objective((const double *)fdat, 1, d, -1.0, (const double *)pen,
                               f_s.dev ? (double *)f_s.dev : (double *)fsum, ctx->stream));
    if (which & 2)
        CK(launch_unpack_theta((const float *)G, d, (float *)gh_s.dev, (float *)gJ_s.dev,
                               ctx->stream));
    CK(copy_back(ctx, f_s));
    CK(copy_back(ctx, gh_s));
    CK(copy_back(ctx, gJ_s));
    if (prec == PLM_SPLIT_BF16) {
        CK(cudaMemcpyAsync(ctx->host_counters + 10, tcflag, sizeof(int), cudaMemcpyDeviceToHost,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (ctx->host_counters[10])
            return fail(ctx, PLM_ETIMEOUT, "tensor-core pipeline wait timed out (code 0x%x)",
                        ctx->host_counters[10]);
    } else if (f_s.host || gh_s.host || gJ_s.host) {
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return PLM_OK;
}

plm_status plm_solve(plm_ctx *ctx, const int8_t *msa, int B, int N, int q,
                     const plm_opts *opts, float *h_out, float *J_out,
                     plm_report *report)
{
    plm_family fam;
    fam.msa = msa;
    fam.B = B;
    fam.N = N;
    fam.h_out = h_out;
    fam.J_out = J_out;
    return plm_solve_batch(ctx, &fam, 1, q, opts, report);
}

static plm_status solve_families(plm_ctx *ctx, const plm_family *fams, int nfam, int q,
                                 const plm_opts *opts, plm_report *reports, bool symmetric);

plm_status plm_solve_batch(plm_ctx *ctx, const plm_family *fams, int nfam, int q,
                           const plm_opts *opts, plm_report *reports)
{
    return solve_families(ctx, fams, nfam, q, opts, reports, false);
}

plm_status plm_solve_symmetric(plm_ctx *ctx, const int8_t *msa, int B, int N, int q,
                               const plm_opts *opts, float *h_out, float *J_out,
                               plm_report *report)
{
    plm_family fam;
    fam.msa = msa;
    fam.B = B;
    fam.N = N;
    fam.h_out = h_out;
    fam.J_out = J_out;
    return solve_families(ctx, &fam, 1, q, opts, report, true);
}

static plm_status solve_families(plm_ctx *ctx, const plm_family *fams, int nfam, int q,
                                 const plm_opts *opts, plm_report *reports, bool symmetric)
{
    if (!ctx) return PLM_EINVAL;
    if (!fams || nfam < 1) return fail(ctx, PLM_EINVAL, "need at least one family");
    for (int f = 0; f < nfam; ++f) {
        plm_status s = check_common(ctx, fams[f].B, fams[f].N, q);
        if (s) return s;
        if (!fams[f].msa) return fail(ctx, PLM_EINVAL, "family %d: msa is NULL", f);
    }
    plm_opts o;
    if (opts) o = *opts;
    else plm_default_opts(&o);
    plm_status s = check_opts(ctx, o);
    if (s) return s;
    CK(cudaSetDevice(ctx->device));
    Problem P;
    P.symmetric = symmetric;
    std::vector<SolveOut> out(nfam);
    std::vector<Staged> hs(nfam), Js(nfam);
    char name[64];
    for (int f = 0; f < nfam; ++f) {
        const int B = fams[f].B, N = fams[f].N;
        const size_t NQ = (size_t)N * Q;
        const void *msa_d;
        snprintf(name, sizeof name, "in_msa_%d", f);
        CK(stage_in(ctx, name, fams[f].msa, (size_t)B * N, &msa_d));
        snprintf(name, sizeof name, "out_h_%d", f);
        CK(stage_out(ctx, name, fams[f].h_out, NQ * sizeof(float), &hs[f]));
        snprintf(name, sizeof name, "out_J_%d", f);
        CK(stage_out(ctx, name, fams[f].J_out, NQ * NQ * sizeof(float), &Js[f]));
        Fam F;
        F.msa = (const int8_t *)msa_d;
        F.d = make_dims(B, N);
        P.fam.push_back(F);
        P.autotune = o.autotune != 0;
        out[f].h = (float *)hs[f].dev;
        out[f].J = (float *)Js[f].dev;
    }
    std::vector<plm_report> reps;
    s = solve_core(ctx, P, o, out, reps);
    if (s) return s;
    for (int f = 0; f < nfam; ++f) {
        CK(copy_back(ctx, hs[f]));
        CK(copy_back(ctx, Js[f]));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    int notconv = 0, noise = 0, total = 0;
    for (int f = 0; f < nfam; ++f) {
        if (reports) reports[f] = reps[f];
        notconv += reps[f].n_noise + reps[f].n_failed;
        noise += reps[f].n_noise;
        total += fams[f].N;
    }
    if (notconv)
        return fail(ctx, PLM_ENOTCONV, "%d of %d sites stopped before gtol (%d at the noise floor)",
                    notconv, total, noise);
    return PLM_OK;
}

plm_status fn_apc_scores(plm_ctx *ctx, const float *J, int N, int q,
                         int combine, double *fn_out, double *cfn_out,
                         int32_t *topL_out, int L, int min_sep)
{
    plm_score_opts so;
    plm_default_score_opts(&so);
    so.combine = combine;
    return plm_scores(ctx, J, N, q, &so, nullptr, fn_out, cfn_out, topL_out, L, min_sep);
}

void plm_default_score_opts(plm_score_opts *so)
{
    if (!so) return;
    memset(so, 0, sizeof *so);
    so->combine = 0;
    so->norm = PLM_NORM_FROBENIUS;
    so->p = 2.0;
    so->exclude_gap = 0;
    so->correction = PLM_CORR_APC;
}

plm_status plm_scores(plm_ctx *ctx, const float *J, int N, int q, const plm_score_opts *opts,
                      const double *freq, double *score_out, double *corr_out,
                      int32_t *topL_out, int L, int min_sep)
{
    if (!ctx) return PLM_EINVAL;
    if (q != Q) return fail(ctx, PLM_EINVAL, "q must be %d (got %d)", Q, q);
    if (N < 2) return fail(ctx, PLM_EINVAL, "N must be >= 2");
    if (!J) return fail(ctx, PLM_EINVAL, "J is NULL");
    if (L < 0 || min_sep < 1) return fail(ctx, PLM_EINVAL, "need L >= 0 and min_sep >= 1");
    if (L > 8192) return fail(ctx, PLM_EINVAL, "L must be <= 8192 (got %d)", L);
    plm_score_opts so;
    if (opts) so = *opts;
    else plm_default_score_opts(&so);
    if (so.combine < 0 || so.combine > 2) return fail(ctx, PLM_EINVAL, "combine must be 0, 1 or 2");
    if (so.norm < PLM_NORM_FROBENIUS || so.norm > PLM_NORM_BURKOFF)
        return fail(ctx, PLM_EINVAL, "unknown norm %d", so.norm);
    if (so.norm == PLM_NORM_LP && !(so.p > 0.0 && std::isfinite(so.p)))
        return fail(ctx, PLM_EINVAL, "the l_p exponent must be > 0");
    if (so.norm == PLM_NORM_BURKOFF && !freq)
        return fail(ctx, PLM_EINVAL, "Burkoff's score needs the site frequencies");
    if (so.norm == PLM_NORM_BURKOFF && so.exclude_gap)
        return fail(ctx, PLM_EINVAL, "gap exclusion applies to the norms only");
    if (so.correction < PLM_CORR_APC || so.correction > PLM_CORR_NONE)
        return fail(ctx, PLM_EINVAL, "unknown correction %d", so.correction);
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const size_t NQ = (size_t)N * Q;
    const void *J_d, *f_d = nullptr;
    CK(stage_in(ctx, "in_J", J, NQ * NQ * sizeof(float), &J_d));
    if (so.norm == PLM_NORM_BURKOFF) CK(stage_in(ctx, "in_freq", freq, NQ * sizeof(double), &f_d));
    Staged fn_s, cfn_s, top_s;
    CK(stage_out(ctx, "out_fn", score_out, (size_t)N * N * sizeof(double), &fn_s));
    CK(stage_out(ctx, "out_cfn", corr_out, (size_t)N * N * sizeof(double), &cfn_s));
    CK(stage_out(ctx, "out_top", topL_out, (size_t)L * 2 * sizeof(int32_t), &top_s));
    void *fn = fn_s.dev, *cfn = cfn_s.dev, *work;
    if (!fn) CK(ws(ctx, "fn", (size_t)N * N * sizeof(double), &fn));
    if (!cfn) CK(ws(ctx, "cfn", (size_t)N * N * sizeof(double), &cfn));
    CK(ws(ctx, "apc_work", ((size_t)N + 1) * sizeof(double), &work));
    ScoreKind sk;
    sk.kind = so.norm;
    sk.p = so.p;
    sk.exclude_gap = so.exclude_gap ? 1 : 0;
    sk.freq = (const double *)f_d;
    {
        ProfScope ps(ctx, "fn_apc_topL");
        CK(launch_fn((const float *)J_d, N, so.combine, (double *)fn, st, sk));
        CK(launch_apc((const double *)fn, N, (double *)cfn, (double *)work, st, so.correction));
        if (top_s.dev) {
            void *tsc;
            CK(ws(ctx, "topL_scratch", topL_scratch_bytes(L), &tsc));
            CK(launch_topL((const double *)cfn, N, L, min_sep, (int32_t *)top_s.dev, tsc, st));
        }
    }
    CK(copy_back(ctx, fn_s));
    CK(copy_back(ctx, cfn_s));
    CK(copy_back(ctx, top_s));
    if (fn_s.host || cfn_s.host || top_s.host) CK(cudaStreamSynchronize(st));
    return PLM_OK;
}

plm_status plmdca_run(plm_ctx *ctx, const int8_t *msa, int B, int N, int q,
                      const plm_opts *opts, int L, int min_sep, float *h_out, float *J_out,
                      double *fn_out, double *cfn_out, int32_t *topL_out, plm_report *report)
{
    if (!ctx) return PLM_EINVAL;
    plm_status s = check_common(ctx, B, N, q);
    if (s) return s;
    CK(cudaSetDevice(ctx->device));
    const size_t NQ = (size_t)N * Q;
    // the couplings stay on the device between the solve and the scores
    Staged hs, Js;
    CK(stage_out(ctx, "run_h", h_out, NQ * sizeof(float), &hs));
    CK(stage_out(ctx, "run_J", J_out, NQ * NQ * sizeof(float), &Js));
    if (!hs.dev) CK(ws(ctx, "run_h", NQ * sizeof(float), &hs.dev));
    if (!Js.dev) CK(ws(ctx, "run_J", NQ * NQ * sizeof(float), &Js.dev));
    plm_family fam;
    fam.msa = msa;
    fam.B = B;
    fam.N = N;
    fam.h_out = (float *)hs.dev;
    fam.J_out = (float *)Js.dev;
    const plm_status st = solve_families(ctx, &fam, 1, q, opts, report, false);
    if (st != PLM_OK && st != PLM_ENOTCONV) return st;
    s = plm_scores(ctx, (const float *)Js.dev, N, q, nullptr, nullptr, fn_out, cfn_out, topL_out,
                   L, min_sep);
    if (s) return s;
    CK(copy_back(ctx, hs));
    CK(copy_back(ctx, Js));
    if (hs.host || Js.host) CK(cudaStreamSynchronize(ctx->stream));
    return st;
}

plm_status msa_frequencies(plm_ctx *ctx, const int8_t *msa, const float *w, double beff, int B,
                           int N, int q, double *f_out)
{
    if (!ctx) return PLM_EINVAL;
    plm_status s = check_common(ctx, B, N, q);
    if (s) return s;
    if (!msa || !w || !f_out) return fail(ctx, PLM_EINVAL, "msa, w and f_out are required");
    if (!(beff > 0.0)) return fail(ctx, PLM_EINVAL, "beff must be > 0");
    CK(cudaSetDevice(ctx->device));
    const void *msa_d, *w_d;
    CK(stage_in(ctx, "in_msa", msa, (size_t)B * N, &msa_d));
    s = check_msa(ctx, (const int8_t *)msa_d, B, N);
    if (s) return s;
    CK(stage_in(ctx, "in_w", w, (size_t)B * sizeof(float), &w_d));
    Staged f_s;
    CK(stage_out(ctx, "out_freq", f_out, (size_t)N * Q * sizeof(double), &f_s));
    CK(launch_site_freqs((const int8_t *)msa_d, (const float *)w_d, B, N, beff,
                         (double *)f_s.dev, ctx->stream));
    CK(copy_back(ctx, f_s));
    if (f_s.host) CK(cudaStreamSynchronize(ctx->stream));
    return PLM_OK;
}

}  // extern "C"
