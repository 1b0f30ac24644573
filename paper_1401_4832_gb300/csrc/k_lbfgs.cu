// k_lbfgs.cu -- batched per-site L-BFGS for step 3 of the rundown.
//
// Every site r minimises its own g_r^(reg) (Eq. g_regdef2) over the row
// block Theta[r] (Eq. npll_2: the N problems are independent); the paper
// names limited-memory BFGS as the minimiser (Sec. 5) and starts at the
// origin (Sec. 6).  All sites share each objective+gradient evaluation; a
// site keeps its own curvature pairs, step length and stopping state.
//
// One CTA per site streams that site's contiguous segment of the vectors
// (FP32 storage); every inner product and every scalar of the recursion and
// of the line search is FP64, reduced in a fixed order.
//
// Direction: the two-loop recursion (Nocedal & Wright, Alg. 7.4) with
// H0 = (s'y / y'y) I.  Step: a strong-Wolfe search (c1, c2) in the style of
// Nocedal & Wright Alg. 3.5/3.6, driven by the directional derivative: the
// objective is convex, so phi'(alpha) is nondecreasing and brackets the
// minimiser along the line even where FP32 rounding makes differences of f
// unresolvable.  The sufficient-decrease test allows a noise band of
// `noise * max(1, |f0|)` on f.
#include "plm_device.cuh"
#include "plm_internal.cuh"

namespace plm {

namespace {

constexpr int LB_THREADS = 512;

__device__ __forceinline__ double dot4(const float4 a, const float4 b)
{
    return (double)a.x * b.x + (double)a.y * b.y + (double)a.z * b.z +
           (double)a.w * b.w;
}

__global__ void __launch_bounds__(LB_THREADS)
k_init(SiteState *ss, const double *__restrict__ f, const float *__restrict__ g,
       Dims d, SolveParams p)
{
    __shared__ double red[LB_THREADS / 32];
    const int r = blockIdx.x;
    const size_t n4 = d.site_elems() / 4;
    const float4 *g4 = (const float4 *)(g + (size_t)r * d.site_elems());
    double gg = 0.0;
    for (size_t e = threadIdx.x; e < n4; e += blockDim.x) {
        float4 v = g4[e];
        gg += dot4(v, v);
    }
    gg = block_sum_d(gg, red);
    if (threadIdx.x == 0) {
        SiteState &s = ss[r];
        s.f = f[r];
        s.gnorm2 = gg;
        s.hist = 0;
        s.head = 0;
        s.iters = 0;
        s.trials = 0;
        s.phase = 0;
        s.gamma = 1.0;
        s.status = (sqrt(gg) <= p.gtol) ? SITE_CONVERGED
                   : (p.max_iter <= 0 ? SITE_FAILED : SITE_READY);
    }
}

// d = -H g by the two-loop recursion; sets up the line search.
__global__ void __launch_bounds__(LB_THREADS)
k_direction(SiteState *ss, const float *__restrict__ g, float *__restrict__ dir,
            const float *__restrict__ S_hist, const float *__restrict__ Y_hist,
            Dims d, SolveParams p)
{
    __shared__ double red[LB_THREADS / 16];
    __shared__ double alph[MAX_M];
    const int r = blockIdx.x;
    SiteState &s = ss[r];
    if (s.status != SITE_READY) return;
    const size_t seg = d.site_elems();
    const size_t n4 = seg / 4;
    const size_t vec = d.theta_elems();  // stride between history slots
    const int m = p.m;
    const int hist = s.hist, head = s.head;
    const float4 *g4 = (const float4 *)(g + (size_t)r * seg);
    float4 *q4 = (float4 *)(dir + (size_t)r * seg);
    auto S4 = [&](int j) { return (const float4 *)(S_hist + (size_t)j * vec + (size_t)r * seg); };
    auto Y4 = [&](int j) { return (const float4 *)(Y_hist + (size_t)j * vec + (size_t)r * seg); };

    double dg0 = 0.0;
    if (hist == 0) {
        double gd = 0.0;
        for (size_t e = threadIdx.x; e < n4; e += blockDim.x) {
            float4 v = g4[e];
            q4[e] = make_float4(-v.x, -v.y, -v.z, -v.w);
            gd -= dot4(v, v);
        }
        dg0 = block_sum_d(gd, red);
    } else {
        // newest .. oldest: slot j_t = (head - 1 - t) mod m
        int j0 = (head - 1 + m) % m;
        double t0 = 0.0;
        {
            const float4 *s0 = S4(j0);
            for (size_t e = threadIdx.x; e < n4; e += blockDim.x) t0 += dot4(s0[e], g4[e]);
        }
        t0 = block_sum_d(t0, red);
        if (threadIdx.x == 0) alph[j0] = s.rho[j0] * t0;
        __syncthreads();
        double carry = 0.0;  // dot computed in the previous pass
        for (int t = 0; t < hist; ++t) {
            const int j = (head - 1 - t + 2 * m) % m;
            const float a = (float)alph[j];
            const float4 *y = Y4(j);
            const bool last = (t + 1 == hist);
            const int jn = (head - 2 - t + 2 * m) % m;
            const float4 *nxt = last ? Y4(j) : S4(jn);
            const float4 *src = (t == 0) ? g4 : q4;
            double acc = 0.0;
            for (size_t e = threadIdx.x; e < n4; e += blockDim.x) {
                float4 v = src[e], yy = y[e];
                v.x -= a * yy.x; v.y -= a * yy.y; v.z -= a * yy.z; v.w -= a * yy.w;
                q4[e] = v;
                acc += dot4(nxt[e], v);
            }
            acc = block_sum_d(acc, red);
            if (!last) {
                if (threadIdx.x == 0) alph[jn] = s.rho[jn] * acc;
                __syncthreads();
            } else {
                carry = acc;  // y_oldest . q
            }
        }
        // second loop, oldest .. newest, starting from r = gamma q
        const double gamma = s.gamma;
        carry *= gamma;
        for (int t = hist - 1; t >= 0; --t) {
            const int j = (head - 1 - t + 2 * m) % m;
            const double beta = s.rho[j] * carry;
            const float coef = (float)(alph[j] - beta);
            const float4 *sj = S4(j);
            const bool first = (t == hist - 1);
            const bool last = (t == 0);
            const int jn = (head - t + 2 * m) % m;  // next newer slot
            const float sc = first ? (float)gamma : 1.0f;
            double acc = 0.0;
            for (size_t e = threadIdx.x; e < n4; e += blockDim.x) {
                float4 v = q4[e], sv = sj[e];
                v.x = sc * v.x + coef * sv.x;
                v.y = sc * v.y + coef * sv.y;
                v.z = sc * v.z + coef * sv.z;
                v.w = sc * v.w + coef * sv.w;
                if (last) {
                    v = make_float4(-v.x, -v.y, -v.z, -v.w);
                    acc += dot4(g4[e], v);
                } else {
                    acc += dot4(Y4(jn)[e], v);
                }
                q4[e] = v;
            }
            acc = block_sum_d(acc, red);
            carry = acc;
        }
        dg0 = carry;  // g . d
        if (!(dg0 < 0.0)) {
            // not a descent direction (rounding): drop the history, use -g
            double gd = 0.0;
            for (size_t e = threadIdx.x; e < n4; e += blockDim.x) {
                float4 v = g4[e];
                q4[e] = make_float4(-v.x, -v.y, -v.z, -v.w);
                gd -= dot4(v, v);
            }
            dg0 = block_sum_d(gd, red);
            if (threadIdx.x == 0) {
                s.hist = 0;
                s.head = 0;
            }
        }
    }
    if (threadIdx.x == 0) {
        s.f0 = s.f;
        s.dg0 = dg0;
        s.alpha = (s.iters == 0 && s.hist == 0) ? 1.0 / sqrt(s.gnorm2) : 1.0;
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

// theta_t = theta + alpha d (and its bf16 hi/lo split); penalty at theta_t
__global__ void __launch_bounds__(LB_THREADS)
k_trial(SiteState *ss, const float *__restrict__ theta,
        const float *__restrict__ dir, float *__restrict__ theta_t,
        __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo,
        Dims d, SolveParams p)
{
    __shared__ double red[LB_THREADS / 16];
    const int r = blockIdx.x;
    SiteState &s = ss[r];
    if (s.status != SITE_SEARCHING) return;
    const size_t seg = d.site_elems();
    const size_t n4 = seg / 4;
    const int NQ = d.N * Q;
    const float a = (float)s.alpha;
    const float4 *t4 = (const float4 *)(theta + (size_t)r * seg);
    const float4 *d4 = (const float4 *)(dir + (size_t)r * seg);
    float4 *o4 = (float4 *)(theta_t + (size_t)r * seg);
    double pj = 0.0, ph = 0.0;
    for (size_t e = threadIdx.x; e < n4; e += blockDim.x) {
        float4 t = t4[e], dv = d4[e];
        float4 v = make_float4(fmaf(a, dv.x, t.x), fmaf(a, dv.y, t.y),
                               fmaf(a, dv.z, t.z), fmaf(a, dv.w, t.w));
        o4[e] = v;
        const float vv[4] = {v.x, v.y, v.z, v.w};
        const int c0 = (int)((4 * e) % d.KP);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            double x = vv[u];
            if (c0 + u == NQ) ph += x * x;
            else pj += x * x;
        }
        if (hi) {
            size_t base = (size_t)r * seg + 4 * e;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                __nv_bfloat16 h = __float2bfloat16_rn(vv[u]);
                hi[base + u] = h;
                lo[base + u] = __float2bfloat16_rn(vv[u] - __bfloat162float(h));
            }
        }
    }
    block_sum2_d(pj, ph, red);
    if (threadIdx.x == 0) s.pen_t = p.lambda_h * ph + p.lambda_Jp * pj;
}

__device__ double safe_interp(double lo, double flo, double dlo, double hi,
                              double fhi, double dhi)
{
    // minimiser of the cubic through (lo, flo, dlo) and (hi, fhi, dhi),
    // kept inside the middle 80% of the interval; bisection otherwise
    double a = lo, b = hi;
    double d1 = dlo + dhi - 3.0 * (flo - fhi) / (a - b);
    double disc = d1 * d1 - dlo * dhi;
    double L = fmin(a, b), H = fmax(a, b);
    if (disc >= 0.0 && isfinite(disc)) {
        double d2 = sqrt(disc);
        if (b < a) d2 = -d2;
        double den = dhi - dlo + 2.0 * d2;
        if (den != 0.0) {
            double t = b - (b - a) * (dhi + d2 - d1) / den;
            double mg = 0.1 * (H - L);
            if (isfinite(t) && t >= L + mg && t <= H - mg) return t;
        }
    }
    // secant on the derivative (phi' is monotone for a convex objective)
    if (dlo < 0.0 && dhi > 0.0) {
        double t = a - dlo * (b - a) / (dhi - dlo);
        double mg = 0.1 * (H - L);
        if (isfinite(t) && t >= L + mg && t <= H - mg) return t;
    }
    return 0.5 * (a + b);
}

enum { LS_CONTINUE = 0, LS_ACCEPT = 1, LS_FAIL = 2 };

// consumes the evaluation at theta_t; one thread per site makes the decision
__global__ void __launch_bounds__(LB_THREADS)
k_linesearch(SiteState *ss, const double *__restrict__ f_data,
             float *__restrict__ theta, float *__restrict__ g,
             const float *__restrict__ theta_t, const float *__restrict__ g_t,
             const float *__restrict__ dir, float *__restrict__ S_hist,
             float *__restrict__ Y_hist, Dims d, SolveParams p,
             int *__restrict__ counters)
{
    __shared__ double red[LB_THREADS / 16];
    __shared__ int action;
    const int r = blockIdx.x;
    SiteState &s = ss[r];
    if (s.status != SITE_SEARCHING) return;
    const size_t seg = d.site_elems();
    const size_t n4 = seg / 4;
    const float4 *gt4 = (const float4 *)(g_t + (size_t)r * seg);
    const float4 *d4 = (const float4 *)(dir + (size_t)r * seg);
    double dgt = 0.0, gn2 = 0.0;
    for (size_t e = threadIdx.x; e < n4; e += blockDim.x) {
        float4 gv = gt4[e];
        dgt += dot4(gv, d4[e]);
        gn2 += dot4(gv, gv);
    }
    block_sum2_d(dgt, gn2, red);

    if (threadIdx.x == 0) {
        const double ft = f_data[r] + s.pen_t;
        const double a = s.alpha, f0 = s.f0, dg0 = s.dg0;
        const double eps = p.noise * fmax(1.0, fabs(f0));
        const bool decrease = (ft <= f0 + p.c1 * a * dg0 + eps) || (dgt <= p.c1 * dg0);
        const bool curv = fabs(dgt) <= p.c2 * fabs(dg0);
        int act = LS_CONTINUE;
        s.trials++;
        if (!isfinite(ft) || !isfinite(dgt)) {
            // step far too long: shrink towards the last good point
            s.a_hi = a;
            s.f_hi = INFINITY;
            s.dg_hi = INFINITY;
            s.phase = 1;
            s.alpha = 0.5 * (s.a_lo + a);
        } else if (decrease && curv) {
            act = LS_ACCEPT;
        } else if (s.phase == 0) {
            if (!decrease || dgt > 0.0) {
                // the minimiser along the line lies in (a_prev, a)
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
        if (act == LS_ACCEPT) {
            s.f = ft;
            s.gnorm2 = gn2;
        } else if (act == LS_FAIL) {
            // a failed search near the optimum is the FP32 noise floor
            s.status = (fabs(ft - f0) <= eps) ? SITE_NOISE : SITE_FAILED;
        }
        action = act;
    }
    __syncthreads();
    if (action == LS_CONTINUE) {
        if (threadIdx.x == 0) atomicAdd(&counters[0], 1);
        return;
    }
    if (action != LS_ACCEPT) return;

    // commit: s = theta_t - theta, y = g_t - g, theta <- theta_t, g <- g_t
    const int slot = s.head;
    const size_t vec = d.theta_elems();
    float4 *th4 = (float4 *)(theta + (size_t)r * seg);
    float4 *g4 = (float4 *)(g + (size_t)r * seg);
    const float4 *tt4 = (const float4 *)(theta_t + (size_t)r * seg);
    float4 *sh4 = (float4 *)(S_hist + (size_t)slot * vec + (size_t)r * seg);
    float4 *yh4 = (float4 *)(Y_hist + (size_t)slot * vec + (size_t)r * seg);
    double sy = 0.0, yy = 0.0;
    for (size_t e = threadIdx.x; e < n4; e += blockDim.x) {
        float4 tn = tt4[e], to = th4[e], gn = gt4[e], go = g4[e];
        float4 sv = make_float4(tn.x - to.x, tn.y - to.y, tn.z - to.z, tn.w - to.w);
        float4 yv = make_float4(gn.x - go.x, gn.y - go.y, gn.z - go.z, gn.w - go.w);
        sh4[e] = sv;
        yh4[e] = yv;
        th4[e] = tn;
        g4[e] = gn;
        sy += dot4(sv, yv);
        yy += dot4(yv, yv);
    }
    block_sum2_d(sy, yy, red);
    if (threadIdx.x == 0) {
        if (sy > 0.0 && yy > 0.0) {
            s.rho[slot] = 1.0 / sy;
            s.gamma = sy / yy;
            s.head = (slot + 1) % p.m;
            if (s.hist < p.m) s.hist++;
        }
        s.iters++;
        if (sqrt(s.gnorm2) <= p.gtol) s.status = SITE_CONVERGED;
        else if (s.iters >= p.max_iter) s.status = SITE_FAILED;
        else s.status = SITE_READY;
    }
}

__global__ void k_count(const SiteState *ss, int N, int *counters)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    int st = ss[r].status;
    if (st == SITE_SEARCHING) atomicAdd(&counters[0], 1);
    if (st == SITE_READY) atomicAdd(&counters[1], 1);
}

}  // namespace

cudaError_t launch_lbfgs_init(SiteState *ss, const double *f, const float *g,
                              const Dims &d, const SolveParams &p,
                              cudaStream_t st)
{
    k_init<<<d.N, LB_THREADS, 0, st>>>(ss, f, g, d, p);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_lbfgs_direction(SiteState *ss, const float *g, float *dir,
                                   const float *S_hist, const float *Y_hist,
                                   const Dims &d, const SolveParams &p,
                                   cudaStream_t st)
{
    k_direction<<<d.N, LB_THREADS, 0, st>>>(ss, g, dir, S_hist, Y_hist, d, p);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_lbfgs_trial(SiteState *ss, const float *theta,
                               const float *dir, float *theta_t,
                               __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                               const Dims &d, const SolveParams &p,
                               cudaStream_t st)
{
    k_trial<<<d.N, LB_THREADS, 0, st>>>(ss, theta, dir, theta_t, hi, lo, d, p);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_lbfgs_linesearch(SiteState *ss, const double *f_data,
                                    float *theta, float *g,
                                    const float *theta_t, const float *g_t,
                                    const float *dir, float *S_hist,
                                    float *Y_hist, const Dims &d,
                                    const SolveParams &p, int *counters,
                                    cudaStream_t st)
{
    k_linesearch<<<d.N, LB_THREADS, 0, st>>>(ss, f_data, theta, g, theta_t, g_t,
                                            dir, S_hist, Y_hist, d, p, counters);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_count_status(const SiteState *ss, int N, int *counters,
                                cudaStream_t st)
{
    k_count<<<(N + 127) / 128, 128, 0, st>>>(ss, N, counters);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace plm
