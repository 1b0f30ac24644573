/*
 * plmdca.h -- C ABI of the GB300 (sm_103a) asymmetric plmDCA library.
 *
 * Method: Ekeberg, Hartonen & Aurell, "Fast pseudolikelihood maximization
 * for direct-coupling analysis of protein structure from many homologous
 * amino-acid sequences" (J. Comput. Phys. 2014).  The calls follow the
 * paper's statement of the problem (Sec. 3.5): an MSA, a reweighting
 * threshold x and regularisation strengths lambda_h, lambda_J go in;
 * couplings and contact scores come out.
 *
 * Conventions for every call
 *   - q must be 21 (20 amino acids + gap, Sec. 2); other values give
 *     PLM_EINVAL.  State 0 is the gap.
 *   - msa is int8 [B][N], row-major (sequence b, position i), values 0..q-1.
 *   - Couplings use the public, unpadded "asymmetric" layout
 *         J[r][s][i][k] = J^r_{ri}(s,k)     (float [N][q][N][q])
 *     i.e. the estimate of coupling (r,i) produced by site r's problem, with
 *     the first state index belonging to r (Sec. 3, remark after Eq.
 *     condpfinal).  Diagonal blocks J[r][.][r][.] are not parameters: they
 *     must be zero on input and are returned zero.  Fields: h[r][s], float
 *     [N][q].
 *   - Array arguments may be device pointers or host pointers (pageable or
 *     pinned); the library checks each with cudaPointerGetAttributes and
 *     stages host arrays through its own device workspace.  The caller keeps
 *     ownership of every array it passes.
 *   - Work is ordered on the context's stream.  Calls that return host
 *     scalars (msa_reweight's B_eff, plm_solve's report) or that were given
 *     host arrays synchronise that stream before returning.
 *   - A status != PLM_OK leaves the outputs unspecified and the context
 *     usable, except PLM_ECUDA after a sticky CUDA error.  plm_last_error()
 *     returns a message for the last failing call on that context.
 *   - Nothing here may be called from two host threads on one context at
 *     the same time.
 */
#ifndef PLMDCA_H
#define PLMDCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct plm_ctx plm_ctx; /* opaque; owns the device workspace */

typedef enum {
    PLM_OK = 0,
    PLM_EINVAL = -1,    /* bad argument (shape, range, null pointer) */
    PLM_ENOMEM = -2,    /* device or host allocation failed */
    PLM_ECUDA = -3,     /* a CUDA call failed */
    PLM_ENOTCONV = -4,  /* plm_solve: some site did not reach gtol */
    PLM_ETIMEOUT = -5,  /* a device-side wait ran out of its budget */
    PLM_ENOTIMPL = -6   /* option not built */
} plm_status;

/* Arithmetic of the two contractions (logits and gradient). */
typedef enum {
    PLM_FP32_EXACT = 0, /* FP32 gather/scatter sums on the CUDA cores */
    PLM_TF32 = 1,       /* reserved; returns PLM_ENOTIMPL */
    PLM_SPLIT_BF16 = 2  /* tcgen05 tensor cores: couplings and residuals split
                           into bf16 hi + lo parts, one-hot operand exact,
                           FP32 accumulation in tensor memory */
} plm_precision;

typedef struct {
    double x;          /* reweighting identity threshold, 0..1 (paper: 0.8) */
    double lambda_h;   /* field strength (paper: 0.01) */
    double lambda_J;   /* coupling strength as the user gives it (paper: 0.01);
                          halved inside, lambda'_J = 0.5 lambda_J (step 1) */
    double gtol;       /* stop a site when ||grad g_r^(reg)||_2 <= gtol */
    int lbfgs_m;       /* L-BFGS memory, 1..8 */
    int max_iter;      /* iteration cap per site */
    int max_ls;        /* trial steps per line search before a site fails */
    plm_precision prec;
    int use_graph;     /* 1: replay the per-iteration launches from CUDA graphs
                          (needs a non-legacy stream) */
    int autotune;      /* 1: time the candidate tensor-core tile shapes once per
                          problem shape (cached for the process) and use the
                          fastest; 0: fixed shapes */
    int reserved[6];
} plm_opts;

typedef struct {
    int iters;         /* iterations of the slowest site */
    int evals;         /* objective+gradient evaluations (all sites each) */
    int n_converged;   /* sites with ||grad|| <= gtol */
    int n_noise;       /* sites stopped because the line search could not
                          resolve a decrease within the FP32 evaluation noise;
                          their gradient norm is reported in gnorm_max */
    int n_failed;      /* sites stopped by max_iter or a failed line search */
    double f_total;    /* sum over sites of g_r^(reg) at the returned point */
    double gnorm_max;  /* largest ||grad g_r^(reg)||_2 over sites */
    double beff;       /* B_eff of the reweighting */
    double seconds;    /* wall time of the call */
} plm_report;

/* Fills opts with the paper's recommended inputs (x = 0.8, lambda_h =
 * lambda_J = 0.01, Sec. 3.5) and gtol = 1e-4, m = 5, max_iter = 1000,
 * max_ls = 20, PLM_SPLIT_BF16, use_graph = 1, autotune = 1. */
void plm_default_opts(plm_opts *opts);

/* Creates a context on CUDA device `device` that orders its work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream). */
plm_status plm_create(plm_ctx **ctx, int device, void *cuda_stream);
plm_status plm_destroy(plm_ctx *ctx);
const char *plm_last_error(plm_ctx *ctx);

/* Step 2 of the rundown, Eq. inverse_weights2 (Sec. 3.1, Eq.
 * inverse_weights): m_b = #{a : similarity(a,b) >= x}, counting b itself and
 * counting a gap facing a gap as identical; similarity >= x is evaluated in
 * integers as matches >= ceil(x N).  w_b = 1/m_b rounded to float, and
 * B_eff = sum_b 1/m_b in double precision (added over the histogram of m in
 * increasing m, so the value is independent of sequence order).
 *   msa      [B][N] int8      in
 *   m_out    [B] int32        out (may be NULL)
 *   w_out    [B] float        out (may be NULL)
 *   beff_out host double      out (may be NULL)
 * Errors: PLM_EINVAL for B < 1, N < 1, x outside [0,1], q != 21, states out
 * of range. */
plm_status msa_reweight(plm_ctx *ctx, const int8_t *msa, int B, int N, int q,
                        double x, int32_t *m_out, float *w_out,
                        double *beff_out);

/* Step 3 of the rundown at one parameter point, all sites at once: the
 * objective g_r^(reg) of Eq. g_regdef2 and its gradient, Eqs. g_gradh2 and
 * g_gradJ2, normalised by 1/B_eff as in the paper:
 *   g_r = -(1/B_eff) sum_b w_b log P(sigma_r^b | sigma_\r^b)
 *         + lambda_h ||h_r||^2 + lambda'_J sum_{i != r} ||J_ri||^2.
 *   w        [B] float        in (from msa_reweight)
 *   beff     B_eff
 *   h, J     in, public layout
 *   lambda_J the user's strength; lambda'_J = 0.5 lambda_J inside (step 1)
 *   prec     PLM_FP32_EXACT or PLM_SPLIT_BF16
 *   f_out    [N] double       out, per-site objective
 *   gh, gJ   out, same layouts as h and J (diagonal blocks zero); both
 *            NULL: the objective only (the gradient contraction is skipped)
 * Errors: PLM_EINVAL for shapes, beff <= 0, negative lambdas, exactly one
 * of gh, gJ NULL. */
plm_status plm_site_objective_grad(plm_ctx *ctx, const int8_t *msa,
                                   const float *w, double beff, int B, int N,
                                   int q, const float *h, const float *J,
                                   double lambda_h, double lambda_J,
                                   plm_precision prec, double *f_out,
                                   float *gh, float *gJ);

/* Steps 1-3 of the rundown: reweighting, then every g_r^(reg) minimised
 * separately (Eq. npll_2) from the origin (Sec. 6) by a batched per-site
 * L-BFGS (Sec. 5 names the method; memory, line search and tolerance come
 * from opts).  All sites share each objective+gradient evaluation; each
 * site keeps its own curvature pairs, step length and stopping state.
 *   h_out [N][q], J_out [N][q][N][q]   out, the asymmetric estimates
 *   report                            out (host, may be NULL)
 * Returns PLM_ENOTCONV (outputs valid) when some site stopped without
 * reaching gtol, PLM_ETIMEOUT if a device wait ran out. */
plm_status plm_solve(plm_ctx *ctx, const int8_t *msa, int B, int N, int q,
                     const plm_opts *opts, float *h_out, float *J_out,
                     plm_report *report);

/* One protein family of a batched solve. */
typedef struct {
    const int8_t *msa;  /* [B][N] int8, states 0..q-1 (device or host) */
    int B, N;
    float *h_out;       /* [N][q] out */
    float *J_out;       /* [N][q][N][q] out, asymmetric estimates */
} plm_family;

/* plm_solve for many independent families of uneven N and B at once (the
 * paper solves families one at a time; this batches them).  Every site of
 * every family is one problem of the same batched L-BFGS; each evaluation
 * covers all families in one launch per kernel (up to 64 families per
 * launch).  The sites' trajectories are the same as in separate plm_solve
 * calls.  reports: [nfam] (host, may be NULL).  Returns PLM_ENOTCONV if any
 * site of any family stopped before gtol (outputs valid). */
plm_status plm_solve_batch(plm_ctx *ctx, const plm_family *fams, int nfam,
                           int q, const plm_opts *opts, plm_report *reports);

/* Symmetric pseudolikelihood maximisation (Sec. 3, Eq. npll_1, with the l2
 * penalty of Eq. l2reg: lambda_h sum ||h_i||^2 + lambda_J sum_{i<j}
 * ||J_ij||^2, lambda_J used as given): one minimisation of l_pseudo + R_l2
 * over the fields and one coupling block per pair, shared by both sites
 * (J_ri = J_ir^T), instead of the N separate problems of plm_solve.
 * Reweighting as in plm_solve; one L-BFGS problem from the origin (memory,
 * line search, max_iter from opts) over the site-contiguous layout
 * restricted to J_ri = J_ir^T, with the gradient projected onto that
 * subspace; stops when the norm of that projected gradient is <= gtol.
 * Same arguments and output layouts as plm_solve; J_out holds both copies
 * of every block (J[j][l][i][k] = J[i][k][j][l]).  The report's site
 * counts all take the one problem's outcome (n_converged = N when it
 * converged).  Returns PLM_ENOTCONV (outputs valid) when it stopped before
 * gtol, PLM_ETIMEOUT if a device wait ran out. */
plm_status plm_solve_symmetric(plm_ctx *ctx, const int8_t *msa, int B, int N, int q,
                               const plm_opts *opts, float *h_out, float *J_out,
                               plm_report *report);

/* Steps 4-6 of the rundown: Ising gauge of every estimate (Eq.
 * gauge_change2), combination of J^i_ij with J^j_ij = (J^j_ji)^T (Eq.
 * average2; combine = 1 / 2 selects the elementwise min / max alternatives
 * of Sec. 6), Frobenius norm (Eq. frob_normtrans2) and the average product
 * correction (Eq. corr_norm2) with ":" = mean over the other N-1
 * positions.  Then the L highest-scoring pairs i<j with j - i >= min_sep,
 * ordered by score descending, ties by (i, j) ascending (Sec. 4 drops pairs
 * with |i-j| <= 4, i.e. min_sep = 5).
 *   J        [N][q][N][q] float   in (asymmetric estimates from plm_solve)
 *   fn_out   [N][N] double        out (may be NULL)
 *   cfn_out  [N][N] double        out (may be NULL)
 *   topL_out [L][2] int32         out (may be NULL); rows beyond the number
 *                                 of eligible pairs are set to -1
 * Errors: PLM_EINVAL for N < 2, q != 21, L < 0 or L > 8192, min_sep < 1,
 * combine outside 0..2. */
plm_status fn_apc_scores(plm_ctx *ctx, const float *J, int N, int q,
                         int combine, double *fn_out, double *cfn_out,
                         int32_t *topL_out, int L, int min_sep);

/* The score alternatives of Sec. 6, on the same combined Ising-gauged
 * blocks as fn_apc_scores:
 *   norm        PLM_NORM_FROBENIUS (Eq. frob_normtrans2, the default),
 *               PLM_NORM_LP: the general l_p norm (sum |J(k,l)|^p)^(1/p)
 *               (Sec. 6 (i); absolute values), exponent p > 0,
 *               PLM_NORM_BURKOFF: Burkoff's D_ij (Sec. 6 (ii), Eqs.
 *               burkoffscore1-2) from the site frequencies freq;
 *   exclude_gap the gap state 0 left out of the norm (Sec. 6 (iii); norms
 *               only);
 *   correction  PLM_CORR_APC (Eq. corr_norm2, the default), PLM_CORR_ASC:
 *               average sum correction S_ij = FN_ij - FN_:j - FN_i: + FN_::
 *               (Sec. 6 (iv), Eq. corr_normsum), PLM_CORR_NONE;
 *   combine     as in fn_apc_scores. */
enum { PLM_NORM_FROBENIUS = 0, PLM_NORM_LP = 1, PLM_NORM_BURKOFF = 2 };
enum { PLM_CORR_APC = 0, PLM_CORR_ASC = 1, PLM_CORR_NONE = 2 };
typedef struct {
    int combine;      /* 0 mean, 1 min, 2 max */
    int norm;         /* PLM_NORM_* */
    double p;         /* l_p exponent */
    int exclude_gap;  /* 0/1 */
    int correction;   /* PLM_CORR_* */
    int reserved[4];
} plm_score_opts;

/* Defaults: mean, Frobenius, p = 2, gap included, APC (= fn_apc_scores). */
void plm_default_score_opts(plm_score_opts *opts);

/* Scores with the chosen variant.  J, score_out, corr_out, topL_out as in
 * fn_apc_scores (score_out = the uncorrected pair score, corr_out = the
 * corrected one the top-L list ranks); freq [N][q] double: the site
 * frequencies (msa_frequencies), required for PLM_NORM_BURKOFF, else
 * unused (may be NULL).  opts NULL = defaults.  Errors: PLM_EINVAL for an
 * unknown norm or correction, p <= 0, Burkoff without freq or with
 * exclude_gap, and as fn_apc_scores. */
plm_status plm_scores(plm_ctx *ctx, const float *J, int N, int q, const plm_score_opts *opts,
                      const double *freq, double *score_out, double *corr_out,
                      int32_t *topL_out, int L, int min_sep);

/* The whole rundown (steps 1-6) in one call: plm_solve, then fn_apc_scores
 * on the estimates while they are still on the device (one upload of the
 * MSA and one download of each result when the buffers are on the host).
 * Arguments as plm_solve and fn_apc_scores (L top pairs, min_sep; any
 * output may be NULL except that the estimates are always computed).
 * Returns PLM_ENOTCONV (outputs valid) as plm_solve does. */
plm_status plmdca_run(plm_ctx *ctx, const int8_t *msa, int B, int N, int q,
                      const plm_opts *opts, int L, int min_sep, float *h_out, float *J_out,
                      double *fn_out, double *cfn_out, int32_t *topL_out, plm_report *report);

/* An aligned protein family as the int8 MSA of the other calls (host code;
 * no counterpart in the paper's equations: Sec. 4 describes the PFAM
 * alignments it uses).  Insert states (lower-case letters, '.') are
 * removed, as the paper does before DCA; match states map to 0 = gap ('-')
 * and 1..20 = A C D E F G H I K L M N P Q R S T V W Y; O, U, B, Z, X read
 * as the gap.
 *   text, len  the file contents (host)
 *   format     0 auto (Stockholm if the text starts with its header),
 *              1 aligned FASTA / A2M, 2 Stockholm
 *   msa_out    [B][N] int8 (host), or NULL to get B and N only
 *   capacity   bytes available at msa_out
 *   B_out, N_out  out: sequences and match columns
 * ctx may be NULL.  Errors: PLM_EINVAL for an unknown format, characters
 * outside the alphabet, sequences with different numbers of match
 * columns, no sequences, or capacity < B N. */
plm_status msa_parse(plm_ctx *ctx, const char *text, size_t len, int format, int8_t *msa_out,
                     long long capacity, int *B_out, int *N_out);

/* Reweighted single-site frequencies f_i(k) = (1/B_eff) sum_b w_b [S_bi = k]
 * (Sec. 3.1 weights; the f_i of Burkoff's score, Eq. burkoffscore2).
 *   msa [B][N] int8, w [B] float (msa_reweight), beff > 0, f_out [N][q]
 *   double.  Errors: PLM_EINVAL for shapes, states outside 0..q-1, beff <= 0. */
plm_status msa_frequencies(plm_ctx *ctx, const int8_t *msa, const float *w, double beff, int B,
                           int N, int q, double *f_out);

/* msa_reweight_static -- the paper has no counterpart to this call.
 * The same reweighting as msa_reweight (identical m, w and B_eff), for
 * callers that cannot allocate memory when they need it: code running while
 * another component owns the allocator (inside a pool or caching-allocator
 * callback), programs that forbid allocation after start-up, and callers
 * that hold only a raw stream.  It needs no context and calls no cudaMalloc,
 * cudaFree or other allocating routine: its scratch is one file-scope
 * device array of 16 MiB that every GPU loading the library holds until the
 * process exits.  The scratch needed is
 *     round256(20 B ceil(N/32)) + round256(4 B) + round256(4 (B + 1)) + 256
 * bytes; larger problems return PLM_ENOMEM before anything is launched.
 *   msa [B][N] int8, m_out [B] int32 (may be NULL), w_out [B] float (may be
 *   NULL), beff_out: one double -- all DEVICE pointers, owned by the caller.
 *   cuda_stream: the cudaStream_t the work is ordered on (NULL = legacy);
 *   it must belong to the current device (the array used is the current
 *   device's), else PLM_EINVAL.
 * Work is queued on the stream; the call does not synchronise.  States
 * outside 0..20 make *beff_out NaN.  PLM_EINVAL for q != 21, B < 1, N < 1,
 * x outside [0,1], a NULL msa/beff_out or a stream of another device;
 * PLM_ECUDA if a CUDA call fails.  Every call looks up the array's device
 * address (cudaGetSymbolAddress, a host-side lookup) in the current
 * context, so calls after cudaDeviceReset or from another context on the
 * same device use that context's array.  The first call in a context may
 * load the library's device code: make it before any stream capture.
 * Every call shares the array and it keeps the previous call's contents
 * (each call clears what must start at zero), so calls whose work overlaps
 * on the GPU race: order them on one stream. */
plm_status msa_reweight_static(const int8_t *msa, int B, int N, int q, double x,
                               int32_t *m_out, float *w_out, double *beff_out,
                               void *cuda_stream);

/* ---- diagnostics (no counterpart in the paper) ----
 * plm_kernel_launches: number of CUDA kernels this library has launched in
 * this process so far (all contexts).
 * plm_profile: with enable = 1 the context brackets each hot kernel with
 * CUDA events on its stream (a small timing overhead); enable = 0 stops and
 * clears the record.  plm_profile_report writes one line per kernel,
 * "name launches total_ms bytes\n", into buf (NUL-terminated, truncated to
 * len); bytes is the algorithmic HBM traffic of the streaming passes of the
 * L-BFGS (each live site's elements once per vector read or written; 0 for
 * kernels not counted); it synchronises the stream and returns the number
 * of bytes needed. */
long long plm_kernel_launches(void);
/* plm_selftest_wait: a diagnostic, not part of the method.  Runs, on the
 * context's stream, the bounded wait that every tensor-core pipeline stage
 * uses, on a barrier nothing arrives on: after its budget (~2 s at the
 * maximum SM clock) the wait gives up, the kernel records a timeout code in
 * an error word and returns normally.  Returns PLM_ETIMEOUT with the code
 * in *code_out (may be NULL) when that happened — the expected outcome —
 * and the context stays usable; PLM_ECUDA if no timeout was reported. */
plm_status plm_selftest_wait(plm_ctx *ctx, int *code_out);
plm_status plm_profile(plm_ctx *ctx, int enable);
int plm_profile_report(plm_ctx *ctx, char *buf, int len);
/* plm_measure_peak: a diagnostic, not part of the method.  Measures the
 * CUDA cores' throughput of one instruction on the current device, the
 * denominator of an ALU-bound roofline: kind 0 FP32 add, 1 FP32 fused
 * multiply-add (one instruction counted once), 2 FP64 add, 3 32-bit
 * three-input logic op (lop3), 4 population count.  Every thread of a grid
 * of 4 x 256-thread blocks per SM runs 16 independent chains; the best of
 * five launches (after two warm-ups, CUDA events on cuda_stream, NULL =
 * legacy stream) gives *ops_per_s, instructions per second over all
 * threads.  Synchronises the stream.  PLM_EINVAL for an unknown kind or a
 * NULL output; PLM_ECUDA if a CUDA call fails. */
plm_status plm_measure_peak(int kind, void *cuda_stream, double *ops_per_s);

#ifdef __cplusplus
}
#endif
#endif /* PLMDCA_H */
