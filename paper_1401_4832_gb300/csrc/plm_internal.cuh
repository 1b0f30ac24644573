// plm_internal.cuh -- internal layout, per-site state and kernel launchers
// of the GB300 plmDCA library (not part of the public ABI).
//
// Internal parameter layout ("site-contiguous padded", the layout every hot
// kernel reads):
//
//   Theta[r][s][c]   float, r < N sites, s < QP = 24 rows per site, c < KP
//     c <  N*Q  : coupling J_ri(s, k) with i = c / Q, k = c % Q  (Eq. condpfinal)
//     c == N*Q  : field h_r(s)  (a column whose one-hot feature is always 1)
//     c >  N*Q  : zero padding up to KP, a multiple of 64
//   rows s = 21..23 are zero padding (the logits of those rows are masked),
//   and the diagonal block c in [r*Q, r*Q + Q) is zero (not a parameter).
//
// With X[b][c] the one-hot expansion of sequence b (X[b][i*Q+k] = [S_bi == k],
// X[b][N*Q] = 1), the logits of every site are one matrix product,
// L[b][(r,s)] = sum_c X[b][c] Theta[(r,s)][c], and the data part of the
// gradient is the transposed product G[(r,s)][c] = sum_b D[b][(r,s)] X[b][c].
// One site's parameters (q + (N-1) q^2 real entries, Sec. 6) are the
// contiguous row block Theta[r], which the per-site L-BFGS kernels stream.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stddef.h>
#include <stdint.h>

#include <atomic>

namespace plm {

// Raises a kernel's dynamic shared-memory limit on the current device the
// first time a launcher runs there (the attribute is per device; `done`
// holds one bit per device, set once the call succeeded).
inline cudaError_t set_smem_limit_once(const void *kernel, int bytes,
                                       std::atomic<unsigned long long> &done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.fetch_or(bit);
    return e;
}

// running count of kernel launches issued by the library (diagnostics)
void count_launches(int n);

constexpr int Q = 21;     // states: 20 amino acids + gap (Sec. 2)
constexpr int QP = 24;    // rows per site in the padded layout
// sites per 128-row accumulator of the single-CTA gradient kernel: its D^T
// box skips the QP - Q padding rows of every site, so 6 sites fill 126 rows
constexpr int GR_SITES = 6;
constexpr int KALIGN = 64;

struct Dims {
    int B = 0, N = 0;
    int K = 0;     // real columns: N*Q couplings + 1 field
    int KP = 0;    // padded columns
    int R = 0;     // rows: N * QP
    __host__ __device__ size_t site_elems() const { return (size_t)QP * KP; }
    __host__ __device__ size_t theta_elems() const { return (size_t)N * QP * KP; }
};

inline Dims make_dims(int B, int N)
{
    Dims d;
    d.B = B;
    d.N = N;
    d.K = N * Q + 1;
    d.KP = (d.K + KALIGN - 1) / KALIGN * KALIGN;
    d.R = N * QP;
    return d;
}

// Per-site state of the batched L-BFGS (all scalars in FP64).
enum SiteStatus : int {
    SITE_READY = 0,      // has f, g at theta; needs a new direction
    SITE_SEARCHING = 1,  // line search in progress
    SITE_CONVERGED = 2,  // ||g|| <= gtol
    SITE_NOISE = 3,      // line search could not resolve a decrease
    SITE_FAILED = 4,     // max_iter reached or a bad direction
};

constexpr int MAX_M = 8;             // largest L-BFGS memory
constexpr int LB_PART = 4 * MAX_M;   // doubles per (site, chunk) partial record
// partial-record slots written by the commit of an accepted step and read by
// the next direction step of that site: s_new . g_new, y_new . g_old
constexpr int LB_SLOT_SG = LB_PART - 2, LB_SLOT_YG = LB_PART - 1;

struct SiteState {
    double f;        // objective at theta
    double gnorm2;   // ||g||^2 at theta
    double f0, dg0;  // objective and slope at the start of the line search
    double alpha;    // current trial step
    double a_prev, f_prev, dg_prev;
    double a_lo, f_lo, dg_lo, a_hi, f_hi, dg_hi;
    double pen_t;    // penalty at the trial point
    double gamma;    // s'y / y'y of the newest pair
    double SY[MAX_M][MAX_M];  // s_i . y_j by ring slot (entries with i older than or equal to j used)
    double YY[MAX_M][MAX_M];  // y_i . y_j by ring slot
    double cg;                 // direction: d = -(cg g + sum cs_j s_j + sum cy_j y_j)
    double cs[MAX_M], cy[MAX_M];
    double u[MAX_M], v[MAX_M];  // s_j . g and y_j . g at the current g, by ring slot
    int status;
    int phase;       // 0: bracketing, 1: zoom
    int trials;
    int iters;
    int hist, head;  // stored pairs, next ring slot
    int commit_round;  // line-search round whose trial point is committed (-1: none)
    int commit_slot;
    int pad_;
};

struct SolveParams {
    double lambda_h, lambda_Jp;  // lambda'_J = 0.5 lambda_J already applied
    double gtol;
    double c1, c2;
    double noise;                // relative FP32 evaluation noise band of f
    int m;
    int max_iter;
    int max_ls;
};

// ---- reweighting (k_reweight.cu) ----
// scratch: planes [5][B][W] uint32 with W = ceil(N/32), m [B], hist [B+1];
// err (device int, caller-zeroed) gets bit 0 set for states outside 0..20
size_t reweight_scratch_bytes(int B, int N);
// the integer identity threshold of Sec. 3.1 (two sequences are similar
// when at least a fraction x of their N positions match): the smallest
// count T with T / N >= x, computed as ceil(x N - 1e-9)
int identity_threshold(double x, int N);
cudaError_t launch_reweight(const int8_t *msa, int B, int N, int T,
                            int32_t *m_out, float *w_out, double *beff_dev,
                            void *scratch, int *err, cudaStream_t st);

// ---- layout conversion (k_layout.cu) ----
// public (h [N][Q], J [N][Q][N][Q]) -> Theta ; diagonal blocks forced to zero
cudaError_t launch_pack_theta(const float *h, const float *J, const Dims &d,
                              float *theta, cudaStream_t st);
// Theta -> public (h, J); either output may be NULL
cudaError_t launch_unpack_theta(const float *theta, const Dims &d, float *h,
                                float *J, cudaStream_t st);
// per-site penalty lambda_h ||h_r||^2 + lambda'_J sum ||J_ri||^2 (FP64)
cudaError_t launch_penalty(const float *theta, const Dims &d, double lambda_h,
                           double lambda_Jp, double *pen, cudaStream_t st);

// ---- FP32 gather path (k_gather.cu) ----
// `active` (per site, may be NULL = all): row tiles without an active site
// are skipped (their outputs are left as they were)
cudaError_t launch_logits_gather(const int8_t *msa, const float *theta,
                                 const Dims &d, float *L, const uint8_t *active,
                                 cudaStream_t st);
// per-(slice, site) FP64 partial sums of w_b (L[b][r][S_br] - lse); residual
// D[b][(r,s)] = (w_b / B_eff)(P - Y) in FP32
int softmax_slices(const Dims &d);
cudaError_t launch_softmax_resid(const int8_t *msa, const float *w,
                                 double beff, const float *L, const Dims &d,
                                 double *partial, float *D, const uint8_t *active,
                                 cudaStream_t st);
// f[r] = -(sum partial)/B_eff + pen[r]  (pen may be NULL)
cudaError_t launch_finish_objective(const double *partial, int slices,
                                    const Dims &d, double beff,
                                    const double *pen, double *f,
                                    cudaStream_t st);
cudaError_t launch_grad_gather(const int8_t *msa, const float *D,
                               const float *theta, const Dims &d,
                               double lambda_h, double lambda_Jp, float *G,
                               const uint8_t *active, cudaStream_t st);

// ---- L-BFGS (k_lbfgs.cu) ----
// All vectors of the solver (theta, g, d, S, Y ...) are arenas holding the
// padded Theta blocks of every family one after another.  A site is a row
// block of one family; its segment is described by SiteInfo, cut into
// chunks of at most LB_CHUNK4 float4 (ChunkInfo).  Vector kernels run a
// grid of resident CTAs that take the chunks in turn (chunk c goes to CTA
// c mod gridDim) and write FP64 partial sums to part[chunk * LB_PART + k];
// one-warp-per-site kernels reduce a site's chunks in a fixed order, so no
// result depends on the grid size.
constexpr int LB_CHUNK4 = 1024;

struct SiteInfo {
    long long off4;  // float4 offset of the segment in every arena vector
    int len4;        // float4 count streamed: the q state rows (Q * KP / 4)
    int KP;          // padded columns of the family
    int NQ;          // N_f * Q: the field column
    int chunk0;      // first chunk of the site
    int nchunks;
    int family;
    int r;           // site index inside its family
};

struct ChunkInfo {
    int site;
    int e0, e1;  // float4 range inside the site segment
};

// the sites a launch works on: sites s0 .. s0 + nsites - 1 and their chunks
// c0 .. c1 - 1 (site and chunk indices are global: the tables describe the
// whole problem)
struct LbLayout {
    const SiteInfo *si;
    const ChunkInfo *ci;
    int s0, nsites;
    int c0, c1;
    long long vec4;  // float4 stride between history slots (arena size / 4)
};

cudaError_t launch_lbfgs_init(SiteState *ss, const double *f, const float *g,
                              const LbLayout &L, const SolveParams &p, double *part,
                              cudaStream_t st);
// direction d = -H g (compact representation) and line-search set-up
// direction d = -H g of every READY site (compact representation, from the
// S'y_n and Y'y_n the commit pass left in the partial records), the first
// trial point theta_t = theta + alpha d of its line search (and the bf16
// split), and the line-search set-up; sites not READY are skipped
cudaError_t launch_lbfgs_direction(SiteState *ss, const float *g, float *dir,
                                   const float *S_hist, const float *Y_hist, const float *theta,
                                   float *theta_t, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                                   const LbLayout &L, const SolveParams &p, double *part,
                                   int *round_ptr, int *counters, uint8_t *active,
                                   cudaStream_t st);
// later trial points of the searches in progress
cudaError_t launch_lbfgs_trial(SiteState *ss, const float *theta, const float *dir,
                               float *theta_t, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                               const LbLayout &L, double *part, const int *counters,
                               cudaStream_t st);
// consumes f_data[site] (data part of the objective at theta_t) and g_t; the
// decision is taken per site.  counters[0] += #sites still searching,
// counters[1] += #sites that became ready for a new direction.
cudaError_t launch_lbfgs_linesearch(SiteState *ss, const double *f_data, const float *g_t,
                                    const float *dir, const LbLayout &L, const SolveParams &p,
                                    double *part, const int *round_ptr, int *counters,
                                    cudaStream_t st);
// commits the steps accepted in this round: S, Y ring slots, theta <- theta_t,
// g <- g_t, and the inner products the next direction needs
cudaError_t launch_lbfgs_commit(const SiteState *ss, float *theta, float *g,
                                const float *theta_t, const float *g_t, float *S_hist,
                                float *Y_hist, const LbLayout &L, const SolveParams &p,
                                double *part, const int *round_ptr, cudaStream_t st);

// closes a round of a device-side loop (CUDA graph while node): counters[9]
// counts the rounds; the loop goes on while counters[0] + counters[1] > 0,
// counters[4] (tensor-core error) is 0 and fewer than max_rounds ran
cudaError_t launch_round_cond(cudaGraphConditionalHandle h, int *counters, int max_rounds,
                              cudaStream_t st);

// ---- symmetric plmDCA (k_symmetric.cu) ----
// G <- its projection on the layouts with J_ri = J_ir^T: both mirror
// entries replaced by their mean (fields, padding, diagonal untouched)
cudaError_t launch_sym_project(float *G, const Dims &d, cudaStream_t st);
// *out = sum_{r < n} f[r], in site order, FP64
cudaError_t launch_sum_sites(const double *f, int n, double *out, cudaStream_t st);

// ---- scores (k_scores.cu) ----
// the pair score: kind 0 Frobenius norm, 1 general l_p norm (exponent p),
// 2 Burkoff's D_ij (freq: [N][Q] site frequencies); exclude_gap leaves
// state 0 out of the norms
struct ScoreKind {
    int kind = 0;
    double p = 2.0;
    int exclude_gap = 0;
    const double *freq = nullptr;
};
cudaError_t launch_fn(const float *J, int N, int combine, double *fn,
                      cudaStream_t st, ScoreKind sk = ScoreKind());
// correction 0: APC, 1: average sum correction, 2: none
cudaError_t launch_apc(const double *fn, int N, double *cfn, double *work,
                       cudaStream_t st, int correction = 0);
// f[i][k] = (1/B_eff) sum_b w_b [S_bi = k]
cudaError_t launch_site_freqs(const int8_t *msa, const float *w, int B, int N, double beff,
                              double *f, cudaStream_t st);
// top-L pairs (j - i >= min_sep) by score descending, ties (i, j) ascending;
// L <= 8192; rows beyond the number of eligible pairs are -1
size_t topL_scratch_bytes(int L);
cudaError_t launch_topL(const double *score, int N, int L, int min_sep,
                        int32_t *ij, void *scratch, cudaStream_t st);

// ---- tcgen05 split-BF16 path (k_tc.cu) ----
// A batch of families evaluated by one launch of each kernel: the tiles of
// every family form one grid.  Each family's arrays are sub-ranges of the
// solver arenas.
constexpr int MAX_FAM = 64;  // families per launch

struct FamDesc {
    const __nv_bfloat16 *th_hi, *th_lo;  // [R][KP] split theta (the logits' B operand)
    const int8_t *msa;        // [B][N]
    const int8_t *msaT;       // [N+1][BP] transposed, padded (built by launch_tc_prepare)
    const float *w;           // [B]
    const float *theta;       // [R][KP] fp32 (penalty term of the gradient)
    float *G;                 // [R][KP] gradient out
    __nv_bfloat16 *dt_hi, *dt_lo;  // [R][BP] residual, transposed
    double *partial;          // [BP/128][N] objective partials
    double *f_data;           // [N] objective out (data term)
    const uint8_t *active;    // [N] sites to evaluate (NULL = all)
    double inv_beff, beff;
    int B, N, KP, BP, R;
    int tile0_logits, tile0_grad;  // first tile of the family in each grid
    int pad_;
};

struct TcBatch {
    int nfam;
    int ntiles_logits, ntiles_grad;
    FamDesc f[MAX_FAM];
};

// split theta (fp32) into bf16 hi + lo: hi = RN(x), lo = RN(x - hi)
cudaError_t launch_split_theta(const float *theta, size_t n, __nv_bfloat16 *hi,
                               __nv_bfloat16 *lo, cudaStream_t st);
int tc_supported();
// bytes of residual / partial / transposed-MSA scratch of one family
size_t tc_family_scratch_bytes(int B, int N);
int tc_padded_B(int B);
// fills the scratch pointers, tile offsets and msaT of every family
// (launches the transposes); scratch[f] points at tc_family_scratch_bytes
cudaError_t launch_tc_prepare(TcBatch &b, void *const *scratch, cudaStream_t st);
// tile shapes: logits tiles of `lg_sites` sites (24 columns each, even,
// 2..10) x 128 sequences; gradient tiles of `gr_rows` rows (128, or 256 as
// two 128-row accumulators sharing each one-hot operand stage) x `gr_ncols`
// columns (multiple of 32, <= 256)
// lg_pair = 1 or 2: the logits on 2-CTA clusters (256 sequences per tile,
// sites packed 21 columns apart, lg_sites = 4, 8 or 12), pipeline stages of
// 128 (1) or 64 (2) of K
// gr_pair = 1: the gradient on 2-CTA clusters (gr_rows = 256, 128 per CTA)
struct TcConfig {
    int lg_sites = 8;
    int gr_ncols = 256;
    int gr_rows = 128;
    int lg_pair = 0;
    int gr_pair = 0;
};
bool tc_config_valid(const TcConfig &c);
// streaming multiprocessors of the current device (queried once per device)
int num_sms();
// one bounded pipeline wait on a barrier nothing arrives on: ORs a timeout
// code into *err after the wait budget (~2 s) and returns normally
cudaError_t launch_wait_selftest(int *err, cudaStream_t st);
// one evaluation of every family of the batch at its split theta (th_hi/lo):
// f_data (data term) and G (with 2 lambda theta) per family.  which: 1 =
// logits + objective only, 2 = gradient only, 3 = both.
// prof: opaque context pointer for per-kernel event timing (NULL = off)
cudaError_t launch_tc_eval(void *prof, const TcBatch &b, const TcConfig &cfg, double lambda_h,
                           double lambda_Jp, int *err_flag, cudaStream_t st, int which = 3);

}  // namespace plm
