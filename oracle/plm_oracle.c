/*
 * plm_oracle.c -- plain FP64 CPU oracle for asymmetric plmDCA
 * (Ekeberg, Hartonen & Aurell, "Fast pseudolikelihood maximization for
 * direct-coupling analysis of protein structure from many homologous
 * amino-acid sequences", J. Comput. Phys. 2014).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no source with the CUDA
 * library (no headers, no tables, no helpers).
 *
 * Every routine is the paper's definition written out as slowly and
 * plainly as possible, in double precision, with one loop per sum of the
 * equations.  OpenMP is used only across sites in the "all sites" wrappers:
 * the site problems are independent (Sec. 3, Eq. npll_2), which is the
 * paper's own parallel scheme.
 *
 * Layouts (all row-major, unpadded, q states per site):
 *   S  : int8  [B][N]        state of sequence b at position i, 0..q-1
 *                            (state 0 is the gap)
 *   h  : double[N][q]        fields h_r(s)
 *   J  : double[N][q][N][q]  J[r][s][i][k] = J^r_{ri}(s,k), the estimate of
 *                            coupling (r,i) from site r's problem; the first
 *                            state index belongs to r (Sec. 3, remark after
 *                            Eq. condpfinal).  Diagonal blocks J[r][.][r][.]
 *                            are not parameters and are kept zero.
 *
 * Parity status: every function here is pinned by the CPU tests (closed
 * forms, brute force enumeration, finite differences, an independent
 * optimiser, invariances); see the test files for which pin covers what.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ENOTCONV (-4)

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* thread count of the OpenMP loops over sites (timing only; results do not
 * depend on it) */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------
 * Step 2 of the rundown (Eq. inverse_weights2): sequence reweighting.
 *
 * similarity(a,b) = (#positions i with S[a][i] == S[b][i]) / N, where a gap
 * matching a gap counts as the same state (Sec. 3.1 says "one of the amino
 * acids or a gap").  Two sequences are similar when similarity >= x; the
 * comparison is done in integers as matches >= T with T = ceil(x N), the
 * smallest integer count whose fraction reaches x.  The sequence itself is
 * among the a's, so m_b >= 1.
 * ---------------------------------------------------------------------- */
int orc_identity_threshold(double x, int N)
{
    /* smallest integer T with T/N >= x; the 1e-9 guards against x*N being
     * computed a hair above an integer */
    double t = ceil(x * (double)N - 1e-9);
    if (t < 0.0) t = 0.0;
    return (int)t;
}

void orc_reweight(const int8_t *S, int B, int N, int T, int32_t *m,
                  double *w, float *w32, double *beff)
{
    for (int b = 0; b < B; ++b) {
        int count = 0;
        for (int a = 0; a < B; ++a) {
            int matches = 0;
            for (int i = 0; i < N; ++i)
                if (S[(size_t)a * N + i] == S[(size_t)b * N + i]) matches++;
            if (matches >= T) count++;
        }
        m[b] = count;
        w[b] = 1.0 / (double)count;
        w32[b] = 1.0f / (float)count;
    }
    /* B_eff = sum_b w_b = sum_k (#b with m_b = k) / k, added in increasing k
     * so that the value does not depend on the order of the sequences */
    int64_t *hist = (int64_t *)calloc((size_t)B + 1, sizeof(int64_t));
    for (int b = 0; b < B; ++b) hist[m[b]]++;
    double acc = 0.0;
    for (int k = 1; k <= B; ++k)
        if (hist[k]) acc += (double)hist[k] / (double)k;
    free(hist);
    *beff = acc;
}

/* ------------------------------------------------------------------------
 * Step 3 of the rundown: objective g_r^(reg) (Eq. g_regdef2) and its
 * gradient (Eqs. g_gradh2 and g_gradJ2) for one site r.
 *
 *   logit(b,s) = h_r(s) + sum_{i != r} J_ri(s, S[b][i])             (Eq. condpfinal)
 *   P(b,s)     = exp(logit(b,s)) / sum_l exp(logit(b,l))
 *   g_r        = -(1/B_eff) sum_b w_b log P(b, S[b][r])
 *                + lambda_h ||h_r||^2 + lambda'_J sum_{i != r} ||J_ri||^2
 *   dg/dh_r(s)     = -(1/B_eff) sum_b w_b (I[S[b][r]=s] - P(b,s)) + 2 lambda_h h_r(s)
 *   dg/dJ_ri(s,k)  = -(1/B_eff) sum_b w_b I[S[b][i]=k] (I[S[b][r]=s] - P(b,s))
 *                    + 2 lambda'_J J_ri(s,k)
 *
 * h_r is [q]; J_r is [q][N][q] (J_r[s][i][k] = J_ri(s,k)); gh_r and gJ_r
 * (same shapes) may be NULL when only the value is wanted.  The log of the
 * normaliser is taken as max + log(sum exp(. - max)), which is the same
 * number computed without overflow.
 * ---------------------------------------------------------------------- */
double orc_site_objgrad(const int8_t *S, const double *w, double beff, int B,
                        int N, int q, int r, const double *h_r,
                        const double *J_r, double lambda_h, double lambda_Jp,
                        double *gh_r, double *gJ_r)
{
    double *logit = (double *)malloc(sizeof(double) * q);
    double *P = (double *)malloc(sizeof(double) * q);
    const size_t Jr_len = (size_t)q * N * q;
    if (gh_r) memset(gh_r, 0, sizeof(double) * q);
    if (gJ_r) memset(gJ_r, 0, sizeof(double) * Jr_len);

    double loglik = 0.0; /* sum_b w_b log P(b, S[b][r]) */
    for (int b = 0; b < B; ++b) {
        const int8_t *seq = S + (size_t)b * N;
        for (int s = 0; s < q; ++s) {
            double acc = h_r[s];
            for (int i = 0; i < N; ++i) {
                if (i == r) continue;
                acc += J_r[((size_t)s * N + i) * q + seq[i]];
            }
            logit[s] = acc;
        }
        double mx = logit[0];
        for (int s = 1; s < q; ++s)
            if (logit[s] > mx) mx = logit[s];
        double z = 0.0;
        for (int s = 0; s < q; ++s) z += exp(logit[s] - mx);
        double lse = mx + log(z);
        int sr = seq[r];
        loglik += w[b] * (logit[sr] - lse);

        if (gh_r || gJ_r) {
            for (int s = 0; s < q; ++s) P[s] = exp(logit[s] - lse);
            for (int s = 0; s < q; ++s) {
                /* -(w_b/B_eff)(I[sr=s] - P) */
                double d = -(w[b] / beff) * ((sr == s ? 1.0 : 0.0) - P[s]);
                if (gh_r) gh_r[s] += d;
                if (gJ_r)
                    for (int i = 0; i < N; ++i) {
                        if (i == r) continue;
                        gJ_r[((size_t)s * N + i) * q + seq[i]] += d;
                    }
            }
        }
    }

    double pen_h = 0.0, pen_J = 0.0;
    for (int s = 0; s < q; ++s) pen_h += h_r[s] * h_r[s];
    for (int s = 0; s < q; ++s)
        for (int i = 0; i < N; ++i) {
            if (i == r) continue;
            for (int k = 0; k < q; ++k) {
                double v = J_r[((size_t)s * N + i) * q + k];
                pen_J += v * v;
            }
        }
    if (gh_r)
        for (int s = 0; s < q; ++s) gh_r[s] += 2.0 * lambda_h * h_r[s];
    if (gJ_r)
        for (int s = 0; s < q; ++s)
            for (int i = 0; i < N; ++i) {
                if (i == r) continue; /* the diagonal block is not a parameter */
                for (int k = 0; k < q; ++k) {
                    size_t e = ((size_t)s * N + i) * q + k;
                    gJ_r[e] += 2.0 * lambda_Jp * J_r[e];
                }
            }
    free(logit);
    free(P);
    return -loglik / beff + lambda_h * pen_h + lambda_Jp * pen_J;
}

/* all sites at one (h, J): f[N], gh[N][q], gJ[N][q][N][q] (gh/gJ may be NULL).
 * lambda_J is the user's coupling strength; step 1 of the rundown halves it. */
void orc_objgrad_all(const int8_t *S, const double *w, double beff, int B,
                     int N, int q, const double *h, const double *J,
                     double lambda_h, double lambda_J, double *f, double *gh,
                     double *gJ)
{
    const double lambda_Jp = 0.5 * lambda_J; /* step 1 of the rundown */
    const size_t Jr_len = (size_t)q * N * q;
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < N; ++r) {
        f[r] = orc_site_objgrad(S, w, beff, B, N, q, r, h + (size_t)r * q,
                                J + (size_t)r * Jr_len, lambda_h, lambda_Jp,
                                gh ? gh + (size_t)r * q : NULL,
                                gJ ? gJ + (size_t)r * Jr_len : NULL);
    }
}

/* ------------------------------------------------------------------------
 * Minimisation of each g_r^(reg) separately (step 3; Sec. 5 says the
 * minimisations used limited-memory BFGS, Sec. 6 says the start point is
 * the origin).  The paper gives no further settings; this oracle uses the
 * textbook method of Nocedal & Wright, Numerical Optimization (2nd ed.):
 *   - search direction by the two-loop recursion (N&W Alg. 7.4) with
 *     H0 = (s'y / y'y) I from the newest pair, memory m;
 *   - first trial step 1/||g|| on iteration 0 (the direction is -g), 1 after;
 *   - step length by the strong-Wolfe line search of N&W Alg. 3.5 with the
 *     zoom of N&W Alg. 3.6, trial points by cubic interpolation with
 *     bisection as the safeguard; c1 = 1e-4, c2 = 0.9;
 *   - stop when ||grad g_r||_2 <= gtol or after max_iter iterations.
 * The parameter vector of site r is theta = [h_r (q), J_r (q*N*q)].
 * ---------------------------------------------------------------------- */
typedef struct {
    const int8_t *S;
    const double *w;
    double beff;
    int B, N, q, r;
    double lambda_h, lambda_Jp;
    int nevals;
    /* objective and gradient at theta; NULL = the site objective g_r^(reg) */
    double (*fg)(void *self, const double *theta, double *grad);
} orc_site_problem;

static double site_fg(orc_site_problem *p, const double *theta, double *grad)
{
    p->nevals++;
    if (p->fg) return p->fg(p, theta, grad);
    return orc_site_objgrad(p->S, p->w, p->beff, p->B, p->N, p->q, p->r,
                            theta, theta + p->q, p->lambda_h, p->lambda_Jp,
                            grad, grad + p->q);
}

static double dot(const double *a, const double *b, size_t n)
{
    double s = 0.0;
    for (size_t k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

/* minimiser of the cubic that matches phi and phi' at a and b (N&W Eq. 3.59),
 * or the midpoint when the cubic has no usable minimiser inside (a, b). */
static double cubic_step(double a, double fa, double da, double b, double fb,
                         double db)
{
    double d1 = da + db - 3.0 * (fa - fb) / (a - b);
    double disc = d1 * d1 - da * db;
    double lo = a < b ? a : b, hi = a < b ? b : a;
    if (disc >= 0.0) {
        double d2 = sqrt(disc);
        if (b < a) d2 = -d2;
        double denom = db - da + 2.0 * d2;
        if (denom != 0.0) {
            double t = b - (b - a) * (db + d2 - d1) / denom;
            double margin = 0.1 * (hi - lo);
            if (t >= lo + margin && t <= hi - margin) return t;
        }
    }
    return 0.5 * (a + b);
}

/* phi(alpha) = g(x + alpha d).  Fills x_out, g_out, f_out at the accepted
 * step; returns 0 on success, -1 when no acceptable step was found. */
static int wolfe_search(orc_site_problem *p, size_t n, const double *x,
                        double f0, const double *g0, const double *d,
                        double alpha1, double *x_out, double *f_out,
                        double *g_out, double *alpha_out)
{
    const double c1 = 1e-4, c2 = 0.9;
    const int max_trials = 40;
    const double dphi0 = dot(g0, d, n);
    if (!(dphi0 < 0.0)) return -1;

    double a_prev = 0.0, f_prev = f0, d_prev = dphi0;
    double a = alpha1;
    int trials = 0;
    int in_zoom = 0;
    double a_lo = 0, f_lo = 0, d_lo = 0, a_hi = 0, f_hi = 0, d_hi = 0;

    for (;;) {
        if (trials++ >= max_trials) return -1;
        for (size_t k = 0; k < n; ++k) x_out[k] = x[k] + a * d[k];
        double fa = site_fg(p, x_out, g_out);
        double da = dot(g_out, d, n);
        if (!in_zoom) {
            /* N&W Alg. 3.5 */
            if (fa > f0 + c1 * a * dphi0 || (trials > 1 && fa >= f_prev)) {
                a_lo = a_prev; f_lo = f_prev; d_lo = d_prev;
                a_hi = a; f_hi = fa; d_hi = da;
                in_zoom = 1;
            } else if (fabs(da) <= -c2 * dphi0) {
                *f_out = fa; *alpha_out = a;
                return 0;
            } else if (da >= 0.0) {
                a_lo = a; f_lo = fa; d_lo = da;
                a_hi = a_prev; f_hi = f_prev; d_hi = d_prev;
                in_zoom = 1;
            } else {
                a_prev = a; f_prev = fa; d_prev = da;
                a = 2.0 * a; /* extrapolate */
                continue;
            }
        } else {
            /* N&W Alg. 3.6, one trial per pass */
            if (fa > f0 + c1 * a * dphi0 || fa >= f_lo) {
                a_hi = a; f_hi = fa; d_hi = da;
            } else {
                if (fabs(da) <= -c2 * dphi0) {
                    *f_out = fa; *alpha_out = a;
                    return 0;
                }
                if (da * (a_hi - a_lo) >= 0.0) {
                    a_hi = a_lo; f_hi = f_lo; d_hi = d_lo;
                }
                a_lo = a; f_lo = fa; d_lo = da;
            }
            if (fabs(a_hi - a_lo) < 1e-16 * (a_lo > 0 ? a_lo : 1.0)) {
                /* interval collapsed: accept the best point if it decreases f */
                if (f_lo < f0 && a_lo > 0.0) {
                    for (size_t k = 0; k < n; ++k) x_out[k] = x[k] + a_lo * d[k];
                    *f_out = site_fg(p, x_out, g_out);
                    *alpha_out = a_lo;
                    return 0;
                }
                return -1;
            }
        }
        a = cubic_step(a_lo, f_lo, d_lo, a_hi, f_hi, d_hi);
    }
}

/* theta: in = start point (the paper starts at the origin), out = minimiser.
 * Returns the number of iterations taken; *status_out is ORC_OK when the
 * gradient norm reached gtol and ORC_ENOTCONV otherwise. */
static int lbfgs_run(orc_site_problem *pp, size_t n, double gtol, int mem, int max_iter,
                     double *theta, double *f_out, double *gnorm_out, int *nevals_out,
                     int *status_out);

int orc_lbfgs_site(const int8_t *S, const double *w, double beff, int B, int N,
                   int q, int r, double lambda_h, double lambda_Jp,
                   double gtol, int mem, int max_iter, double *theta,
                   double *f_out, double *gnorm_out, int *nevals_out,
                   int *status_out)
{
    orc_site_problem p = {S, w, beff, B, N, q, r, lambda_h, lambda_Jp, 0, NULL};
    const size_t n = (size_t)q + (size_t)q * N * q;
    return lbfgs_run(&p, n, gtol, mem, max_iter, theta, f_out, gnorm_out, nevals_out,
                     status_out);
}

/* the L-BFGS iteration described above, for any objective (pp->fg) */
static int lbfgs_run(orc_site_problem *pp, size_t n, double gtol, int mem, int max_iter,
                     double *theta, double *f_out, double *gnorm_out, int *nevals_out,
                     int *status_out)
{
    orc_site_problem *p = pp;
    double *g = (double *)malloc(sizeof(double) * n);
    double *d = (double *)malloc(sizeof(double) * n);
    double *xn = (double *)malloc(sizeof(double) * n);
    double *gn = (double *)malloc(sizeof(double) * n);
    double *sh = (double *)malloc(sizeof(double) * n * (size_t)mem);
    double *yh = (double *)malloc(sizeof(double) * n * (size_t)mem);
    double *rho = (double *)malloc(sizeof(double) * mem);
    double *alph = (double *)malloc(sizeof(double) * mem);
    int hist = 0, head = 0; /* number of stored pairs, next slot */
    int status = ORC_ENOTCONV, it = 0;

    double f = site_fg(p, theta, g);
    double gnorm = sqrt(dot(g, g, n));
    for (it = 0; it < max_iter; ++it) {
        if (gnorm <= gtol) { status = ORC_OK; break; }
        /* two-loop recursion (N&W Alg. 7.4): d = -H g */
        for (size_t k = 0; k < n; ++k) d[k] = g[k];
        for (int t = 0; t < hist; ++t) {
            int j = (head - 1 - t + mem) % mem; /* newest first */
            alph[j] = rho[j] * dot(sh + (size_t)j * n, d, n);
            for (size_t k = 0; k < n; ++k) d[k] -= alph[j] * yh[(size_t)j * n + k];
        }
        if (hist > 0) {
            int j = (head - 1 + mem) % mem;
            double gamma = dot(sh + (size_t)j * n, yh + (size_t)j * n, n) /
                           dot(yh + (size_t)j * n, yh + (size_t)j * n, n);
            for (size_t k = 0; k < n; ++k) d[k] *= gamma;
        }
        for (int t = hist - 1; t >= 0; --t) {
            int j = (head - 1 - t + mem) % mem; /* oldest first */
            double beta = rho[j] * dot(yh + (size_t)j * n, d, n);
            for (size_t k = 0; k < n; ++k) d[k] += sh[(size_t)j * n + k] * (alph[j] - beta);
        }
        for (size_t k = 0; k < n; ++k) d[k] = -d[k];

        double alpha1 = (it == 0 && hist == 0) ? 1.0 / gnorm : 1.0;
        double fn, alpha;
        if (wolfe_search(p, n, theta, f, g, d, alpha1, xn, &fn, gn, &alpha) != 0) {
            status = ORC_ENOTCONV;
            break;
        }
        /* curvature pair s = x_new - x, y = g_new - g */
        double *s_new = sh + (size_t)head * n, *y_new = yh + (size_t)head * n;
        for (size_t k = 0; k < n; ++k) {
            s_new[k] = xn[k] - theta[k];
            y_new[k] = gn[k] - g[k];
        }
        double sy = dot(s_new, y_new, n);
        if (sy > 0.0) {
            rho[head] = 1.0 / sy;
            head = (head + 1) % mem;
            if (hist < mem) hist++;
        }
        memcpy(theta, xn, sizeof(double) * n);
        memcpy(g, gn, sizeof(double) * n);
        f = fn;
        gnorm = sqrt(dot(g, g, n));
    }
    if (it >= max_iter && gnorm <= gtol) status = ORC_OK;
    if (f_out) *f_out = f;
    if (gnorm_out) *gnorm_out = gnorm;
    if (nevals_out) *nevals_out = p->nevals;
    if (status_out) *status_out = status;
    free(g); free(d); free(xn); free(gn); free(sh); free(yh); free(rho); free(alph);
    return it;
}

/* Solve the sites listed in `sites` (or all N when sites == NULL) from the
 * origin.  h and J are [N][q] and [N][q][N][q]; only the rows of the listed
 * sites are written.  iters/status/f/gnorm/nevals are per listed site. */
void orc_solve_sites(const int8_t *S, const double *w, double beff, int B,
                     int N, int q, double lambda_h, double lambda_J,
                     double gtol, int mem, int max_iter, const int32_t *sites,
                     int nsites, double *h, double *J, int32_t *iters,
                     int32_t *status, double *f, double *gnorm,
                     int32_t *nevals)
{
    const double lambda_Jp = 0.5 * lambda_J; /* step 1 of the rundown */
    const size_t Jr_len = (size_t)q * N * q;
    const int count = sites ? nsites : N;
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < count; ++t) {
        int r = sites ? sites[t] : t;
        size_t n = (size_t)q + Jr_len;
        double *theta = (double *)calloc(n, sizeof(double)); /* origin */
        int st = 0, ne = 0;
        double fr = 0, gr = 0;
        int it = orc_lbfgs_site(S, w, beff, B, N, q, r, lambda_h, lambda_Jp,
                                gtol, mem, max_iter, theta, &fr, &gr, &ne, &st);
        memcpy(h + (size_t)r * q, theta, sizeof(double) * q);
        memcpy(J + (size_t)r * Jr_len, theta + q, sizeof(double) * Jr_len);
        if (iters) iters[t] = it;
        if (status) status[t] = st;
        if (f) f[t] = fr;
        if (gnorm) gnorm[t] = gr;
        if (nevals) nevals[t] = ne;
        free(theta);
    }
}

/* ------------------------------------------------------------------------
 * Symmetric pseudolikelihood maximisation (Sec. 3, Eq. npll_1, with the l2
 * penalty of Eq. l2reg): one minimisation of
 *     l_pseudo(h, J) + R_l2(h, J),   l_pseudo = sum_r g_r(h_r, J_r),
 *     R_l2 = lambda_h sum_i ||h_i||^2 + lambda_J sum_{i<j} ||J_ij||^2,
 * where site r's conditional uses J_ri(s,k) = J_ir(k,s) for i < r, i.e. one
 * coupling block per pair shared by both sites.
 * Parameter vector x = [h (N*q) | J_ij for i < j in the order (0,1), (0,2),
 * ..., (0,N-1), (1,2), ... (q*q each, J_ij[k][l] with k the state of i)].
 * The objective is evaluated through the per-site g_r written above: with
 * lambda' = lambda_J / 2 each block's penalty is counted once from each of
 * its two sites, so sum_r g_r^(reg) = l_pseudo + R_l2 (the remark after
 * Eq. g_reg), and the gradient of a shared block is the sum of its two
 * per-site gradients, the second transposed.
 * ---------------------------------------------------------------------- */
static size_t pair_index(int i, int j, int N) /* i < j */
{
    return (size_t)i * N - (size_t)i * (i + 1) / 2 + (size_t)(j - i - 1);
}

size_t orc_sym_nparams(int N, int q)
{
    return (size_t)N * q + (size_t)N * (N - 1) / 2 * q * q;
}

/* expand x into the per-site layout h[N][q], J[N][q][N][q] (both copies) */
void orc_sym_expand(const double *x, int N, int q, double *h, double *J)
{
    memcpy(h, x, sizeof(double) * N * q);
    const double *xJ = x + (size_t)N * q;
    memset(J, 0, sizeof(double) * (size_t)N * q * N * q);
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            const double *blk = xJ + pair_index(i, j, N) * q * q;
            for (int k = 0; k < q; ++k)
                for (int l = 0; l < q; ++l) {
                    J[(((size_t)i * q + k) * N + j) * q + l] = blk[k * q + l]; /* J_ij(k,l) */
                    J[(((size_t)j * q + l) * N + i) * q + k] = blk[k * q + l]; /* J_ji(l,k) */
                }
        }
}

/* l_pseudo + R_l2 at x; gx (may be NULL) gets its gradient */
double orc_sym_objgrad(const int8_t *S, const double *w, double beff, int B, int N,
                       int q, const double *x, double lambda_h, double lambda_J,
                       double *gx)
{
    const size_t Jlen = (size_t)N * q * N * q;
    double *h = (double *)malloc(sizeof(double) * N * q);
    double *J = (double *)malloc(sizeof(double) * Jlen);
    double *f = (double *)malloc(sizeof(double) * N);
    double *gh = gx ? (double *)malloc(sizeof(double) * N * q) : NULL;
    double *gJ = gx ? (double *)malloc(sizeof(double) * Jlen) : NULL;
    orc_sym_expand(x, N, q, h, J);
    orc_objgrad_all(S, w, beff, B, N, q, h, J, lambda_h, lambda_J, f, gh, gJ);
    double total = 0.0;
    for (int r = 0; r < N; ++r) total += f[r];
    if (gx) {
        memcpy(gx, gh, sizeof(double) * N * q);
        double *gxJ = gx + (size_t)N * q;
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j) {
                double *blk = gxJ + pair_index(i, j, N) * q * q;
                for (int k = 0; k < q; ++k)
                    for (int l = 0; l < q; ++l)
                        blk[k * q + l] = gJ[(((size_t)i * q + k) * N + j) * q + l] +
                                         gJ[(((size_t)j * q + l) * N + i) * q + k];
            }
    }
    free(h); free(J); free(f); free(gh); free(gJ);
    return total;
}

typedef struct {
    orc_site_problem base; /* first member: the L-BFGS driver passes its address */
    double lambda_J;
} orc_sym_problem;

static double sym_fg(void *self, const double *x, double *grad)
{
    orc_sym_problem *p = (orc_sym_problem *)self;
    return orc_sym_objgrad(p->base.S, p->base.w, p->base.beff, p->base.B, p->base.N,
                           p->base.q, x, p->base.lambda_h, p->lambda_J, grad);
}

/* minimise l_pseudo + R_l2 from the origin with the same L-BFGS as the site
 * problems (memory mem, strong Wolfe, stop at ||grad||_2 <= gtol, the
 * gradient in the parameters x); x gets the minimiser */
int orc_solve_symmetric(const int8_t *S, const double *w, double beff, int B, int N, int q,
                        double lambda_h, double lambda_J, double gtol, int mem, int max_iter,
                        double *x, double *f_out, double *gnorm_out, int *nevals_out,
                        int *status_out)
{
    orc_sym_problem p;
    memset(&p, 0, sizeof p);
    p.base.S = S;
    p.base.w = w;
    p.base.beff = beff;
    p.base.B = B;
    p.base.N = N;
    p.base.q = q;
    p.base.lambda_h = lambda_h;
    p.base.fg = sym_fg;
    p.lambda_J = lambda_J;
    const size_t n = orc_sym_nparams(N, q);
    memset(x, 0, sizeof(double) * n); /* origin */
    return lbfgs_run(&p.base, n, gtol, mem, max_iter, x, f_out, gnorm_out, nevals_out,
                     status_out);
}

/* ------------------------------------------------------------------------
 * Step 4 (Eq. gauge_change2): Ising gauge of one q x q block,
 *   Jhat(k,l) = J(k,l) - J(:,l) - J(k,:) + J(:,:)   (":" = mean over states)
 * ---------------------------------------------------------------------- */
void orc_ising_gauge_block(const double *Jb, int q, double *out)
{
    double *rowm = (double *)malloc(sizeof(double) * q);
    double *colm = (double *)malloc(sizeof(double) * q);
    double all = 0.0;
    for (int k = 0; k < q; ++k) {
        double s = 0.0;
        for (int l = 0; l < q; ++l) s += Jb[k * q + l];
        rowm[k] = s / q; /* J(k,:) */
    }
    for (int l = 0; l < q; ++l) {
        double s = 0.0;
        for (int k = 0; k < q; ++k) s += Jb[k * q + l];
        colm[l] = s / q; /* J(:,l) */
    }
    for (int k = 0; k < q; ++k)
        for (int l = 0; l < q; ++l) all += Jb[k * q + l];
    all /= (double)q * q; /* J(:,:) */
    for (int k = 0; k < q; ++k)
        for (int l = 0; l < q; ++l)
            out[k * q + l] = Jb[k * q + l] - colm[l] - rowm[k] + all;
    free(rowm);
    free(colm);
}

/* ------------------------------------------------------------------------
 * Steps 4-6, first half: for every pair i<j take site i's block
 * J^i_ij(k,l) = J[i][k][j][l] and site j's block J^j_ij(k,l) = J^j_ji(l,k)
 * = J[j][l][i][k] (first index belongs to the solving site), move both to
 * the Ising gauge (Eq. gauge_change2), combine them -- average (Eq.
 * average2), or, with combine = 1/2, the elementwise min/max alternatives
 * that Sec. 6 mentions -- and take the Frobenius norm (Eq. frob_normtrans2).
 * fn is [N][N], symmetric, zero on the diagonal.
 * ---------------------------------------------------------------------- */
void orc_fn(const double *J, int N, int q, int combine, double *fn)
{
    const size_t Jr_len = (size_t)q * N * q;
    memset(fn, 0, sizeof(double) * N * N);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < N; ++i) {
        double *bi = (double *)malloc(sizeof(double) * q * q);
        double *bj = (double *)malloc(sizeof(double) * q * q);
        double *gi = (double *)malloc(sizeof(double) * q * q);
        double *gj = (double *)malloc(sizeof(double) * q * q);
        for (int j = i + 1; j < N; ++j) {
            for (int k = 0; k < q; ++k)
                for (int l = 0; l < q; ++l) {
                    bi[k * q + l] = J[(size_t)i * Jr_len + ((size_t)k * N + j) * q + l];
                    bj[k * q + l] = J[(size_t)j * Jr_len + ((size_t)l * N + i) * q + k];
                }
            orc_ising_gauge_block(bi, q, gi);
            orc_ising_gauge_block(bj, q, gj);
            double ss = 0.0;
            for (int e = 0; e < q * q; ++e) {
                double v;
                if (combine == 1) v = gi[e] < gj[e] ? gi[e] : gj[e];
                else if (combine == 2) v = gi[e] > gj[e] ? gi[e] : gj[e];
                else v = 0.5 * (gi[e] + gj[e]);
                ss += v * v;
            }
            fn[(size_t)i * N + j] = sqrt(ss);
            fn[(size_t)j * N + i] = sqrt(ss);
        }
        free(bi); free(bj); free(gi); free(gj);
    }
}

/* Step 6, second half (Eq. corr_norm2): average product correction
 *   S_ij = FN_ij - FN_:j FN_i: / FN_::
 * where ":" is the mean over positions.  The means are over the N-1 true
 * pairs of a row and the N(N-1) ordered pairs overall (the diagonal is not
 * a pair): FN_i: = sum_{j != i} FN_ij / (N-1), FN_:: = sum_{i != j} FN_ij /
 * (N(N-1)).  cfn is [N][N] with a zero diagonal.  When every FN is zero the
 * correction term is 0/0; it is taken as 0 (its limit along any path on which
 * the FN values shrink together). */
void orc_apc(const double *fn, int N, double *cfn)
{
    double *row = (double *)malloc(sizeof(double) * N);
    double *col = (double *)malloc(sizeof(double) * N);
    double tot = 0.0;
    for (int i = 0; i < N; ++i) {
        double s = 0.0;
        for (int j = 0; j < N; ++j)
            if (j != i) s += fn[(size_t)i * N + j];
        row[i] = s / (N - 1);
        tot += s;
    }
    for (int j = 0; j < N; ++j) {
        double s = 0.0;
        for (int i = 0; i < N; ++i)
            if (i != j) s += fn[(size_t)i * N + j];
        col[j] = s / (N - 1);
    }
    tot /= (double)N * (N - 1);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            cfn[(size_t)i * N + j] =
                (i == j) ? 0.0
                         : fn[(size_t)i * N + j] -
                               (tot > 0.0 ? col[j] * row[i] / tot : 0.0);
    free(row);
    free(col);
}

void orc_scores(const double *J, int N, int q, int combine, double *fn,
                double *cfn)
{
    orc_fn(J, N, q, combine, fn);
    orc_apc(fn, N, cfn);
}

/* ------------------------------------------------------------------------
 * The score alternatives of Sec. 6.
 *
 * Reweighted single-site frequencies (Sec. 3.1 weights):
 *     f_i(k) = (1/B_eff) sum_b w_b [S_bi = k]
 * ---------------------------------------------------------------------- */
void orc_site_freqs(const int8_t *S, const double *w, double beff, int B, int N, int q,
                    double *f)
{
    memset(f, 0, sizeof(double) * N * q);
    for (int b = 0; b < B; ++b)
        for (int i = 0; i < N; ++i) f[(size_t)i * q + S[(size_t)b * N + i]] += w[b];
    for (int e = 0; e < N * q; ++e) f[e] /= beff;
}

/* Score of every pair from the combined Ising-gauged block v (the same block
 * orc_fn takes the Frobenius norm of):
 *   kind 0  Frobenius norm (Eq. frob_normtrans2)
 *   kind 1  the general l_p norm (sum_{k,l} |v(k,l)|^p)^(1/p) of Sec. 6 (i)
 *           (absolute values: the l_p norm of the block's entries)
 *   kind 2  Burkoff's score (Sec. 6 (ii), Eqs. burkoffscore1-2):
 *           P(k,l) = f_i(k) f_j(l) e^{v(k,l)} / Z, Z normalising P over k,l,
 *           D_ij = sum_{k,l} P(k,l) ln(P(k,l) / (f_i(k) f_j(l))),
 *           terms with P = 0 (a state never seen) taken as 0
 * exclude_gap (kinds 0, 1): the gap state 0 is left out of the sum
 * (Sec. 6 (iii)).  score is [N][N], symmetric, zero on the diagonal. */
void orc_score_matrix(const double *J, int N, int q, int combine, int kind, double p,
                      int exclude_gap, const double *freq, double *score)
{
    const size_t Jr_len = (size_t)q * N * q;
    memset(score, 0, sizeof(double) * N * N);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < N; ++i) {
        double *bi = (double *)malloc(sizeof(double) * q * q);
        double *bj = (double *)malloc(sizeof(double) * q * q);
        double *gi = (double *)malloc(sizeof(double) * q * q);
        double *gj = (double *)malloc(sizeof(double) * q * q);
        double *v = (double *)malloc(sizeof(double) * q * q);
        for (int j = i + 1; j < N; ++j) {
            for (int k = 0; k < q; ++k)
                for (int l = 0; l < q; ++l) {
                    bi[k * q + l] = J[(size_t)i * Jr_len + ((size_t)k * N + j) * q + l];
                    bj[k * q + l] = J[(size_t)j * Jr_len + ((size_t)l * N + i) * q + k];
                }
            orc_ising_gauge_block(bi, q, gi);
            orc_ising_gauge_block(bj, q, gj);
            for (int e = 0; e < q * q; ++e) {
                if (combine == 1) v[e] = gi[e] < gj[e] ? gi[e] : gj[e];
                else if (combine == 2) v[e] = gi[e] > gj[e] ? gi[e] : gj[e];
                else v[e] = 0.5 * (gi[e] + gj[e]);
            }
            double out = 0.0;
            if (kind == 2) {
                const double *fi = freq + (size_t)i * q, *fj = freq + (size_t)j * q;
                /* P is unchanged when the same constant is taken off every
                 * exponent (Z absorbs it); taking off the block maximum keeps
                 * exp() finite for large couplings */
                double vmax = v[0];
                for (int e = 1; e < q * q; ++e)
                    if (v[e] > vmax) vmax = v[e];
                double Z = 0.0;
                for (int k = 0; k < q; ++k)
                    for (int l = 0; l < q; ++l) Z += fi[k] * fj[l] * exp(v[k * q + l] - vmax);
                for (int k = 0; k < q; ++k)
                    for (int l = 0; l < q; ++l) {
                        double P = fi[k] * fj[l] * exp(v[k * q + l] - vmax) / Z;
                        if (P > 0.0) out += P * log(P / (fi[k] * fj[l]));
                    }
            } else {
                double acc = 0.0;
                for (int k = 0; k < q; ++k)
                    for (int l = 0; l < q; ++l) {
                        if (exclude_gap && (k == 0 || l == 0)) continue;
                        double a = fabs(v[k * q + l]);
                        acc += kind == 1 ? pow(a, p) : a * a;
                    }
                out = kind == 1 ? pow(acc, 1.0 / p) : sqrt(acc);
            }
            score[(size_t)i * N + j] = out;
            score[(size_t)j * N + i] = out;
        }
        free(bi); free(bj); free(gi); free(gj); free(v);
    }
}

/* Average sum correction (Sec. 6 (iv), Eq. corr_normsum):
 *   S_ij = FN_ij - FN_:j - FN_i: + FN_::
 * with the same off-diagonal means as the APC (orc_apc). */
void orc_asc(const double *fn, int N, double *out)
{
    double *row = (double *)malloc(sizeof(double) * N);
    double *col = (double *)malloc(sizeof(double) * N);
    double tot = 0.0;
    for (int i = 0; i < N; ++i) {
        double s = 0.0;
        for (int j = 0; j < N; ++j)
            if (j != i) s += fn[(size_t)i * N + j];
        row[i] = s / (N - 1);
        tot += s;
    }
    for (int j = 0; j < N; ++j) {
        double s = 0.0;
        for (int i = 0; i < N; ++i)
            if (i != j) s += fn[(size_t)i * N + j];
        col[j] = s / (N - 1);
    }
    tot /= (double)N * (N - 1);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            out[(size_t)i * N + j] =
                (i == j) ? 0.0 : fn[(size_t)i * N + j] - col[j] - row[i] + tot;
    free(row);
    free(col);
}

/* Top-L contact list: pairs i<j with j - i >= min_sep ranked by score
 * descending, ties broken by (i, j) ascending.  Returns the number written
 * (min(L, #eligible pairs)); ij is [L][2]. */
int orc_topL(const double *score, int N, int L, int min_sep, int32_t *ij)
{
    int written = 0;
    /* plain selection: repeatedly take the best pair not yet taken */
    char *taken = (char *)calloc((size_t)N * N, 1);
    for (int t = 0; t < L; ++t) {
        int bi = -1, bj = -1;
        double best = 0.0;
        for (int i = 0; i < N; ++i)
            for (int j = i + min_sep; j < N; ++j) {
                if (taken[(size_t)i * N + j]) continue;
                double v = score[(size_t)i * N + j];
                if (bi < 0 || v > best) { best = v; bi = i; bj = j; }
            }
        if (bi < 0) break;
        taken[(size_t)bi * N + bj] = 1;
        ij[2 * t] = bi;
        ij[2 * t + 1] = bj;
        written++;
    }
    free(taken);
    return written;
}
