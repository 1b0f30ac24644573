/*
 * synth_gibbs.c -- seeded Gibbs sampler for synthetic Potts-model MSAs.
 *
 * Input generator only: it draws the sequences that both the CUDA library
 * and the CPU oracle consume.  It computes nothing of the inference method
 * (no weights, no pseudolikelihood, no gradient, no scores).
 *
 * Model: P(sigma) ~ exp(sum_i h_i(sigma_i) + sum_{i<j} J_ij(sigma_i, sigma_j))
 * with a sparse set of coupled pairs, given as a CSR neighbour list where
 * every edge (i -> j) carries the q x q block oriented [state at i][state at j].
 *
 * Each of the B chains starts from a uniformly random sequence and makes
 * `sweeps` systematic-scan sweeps over the sites 0..N-1; site i is redrawn
 * from its conditional distribution given the other sites.  The sample is
 * the final state of the chain.
 *
 * Random numbers: Philox-4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11), keyed by (seed, 0) with the
 * counter (site, sweep, chain, stream); one uniform per draw.  The result
 * therefore does not depend on the number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
    uint32_t v[4];
} philox_ctr;

static inline void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

static philox_ctr philox4x32_10(philox_ctr c, uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int round = 0; round < 10; ++round) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(M0, c.v[0], &hi0, &lo0);
        mulhilo32(M1, c.v[2], &hi1, &lo1);
        philox_ctr n;
        n.v[0] = hi1 ^ c.v[1] ^ k0;
        n.v[1] = lo1;
        n.v[2] = hi0 ^ c.v[3] ^ k1;
        n.v[3] = lo0;
        c = n;
        k0 += W0;
        k1 += W1;
    }
    return c;
}

/* uniform double in [0, 1) from 53 random bits */
static inline double u01(philox_ctr r)
{
    uint64_t x = ((uint64_t)r.v[0] << 21) ^ (uint64_t)(r.v[1] >> 11);
    x &= ((uint64_t)1 << 53) - 1;
    return (double)x * (1.0 / 9007199254740992.0);
}

/* exported for the generator's own unit test (known-answer vectors) */
void synth_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    philox_ctr c = {{ctr[0], ctr[1], ctr[2], ctr[3]}};
    philox_ctr r = philox4x32_10(c, key[0], key[1]);
    for (int k = 0; k < 4; ++k) out[k] = r.v[k];
}

int synth_gibbs(int N, int q, int B, int sweeps, uint32_t seed,
                const double *h,          /* [N][q] */
                const int32_t *nbr_ptr,   /* [N+1] */
                const int32_t *nbr_idx,   /* [E] */
                const double *nbr_blk,    /* [E][q][q] */
                int8_t *out)              /* [B][N] */
{
    if (q > 127 || q < 1) return -1;
#pragma omp parallel
    {
        int8_t *sig = (int8_t *)malloc((size_t)N);
        double *logit = (double *)malloc(sizeof(double) * q);
        double *cum = (double *)malloc(sizeof(double) * q);
#pragma omp for schedule(static)
        for (int b = 0; b < B; ++b) {
            for (int i = 0; i < N; ++i) {
                philox_ctr c = {{(uint32_t)i, 0xFFFFFFFFu, (uint32_t)b, 1u}};
                double u = u01(philox4x32_10(c, seed, 0u));
                int s = (int)(u * q);
                sig[i] = (int8_t)(s < q ? s : q - 1);
            }
            for (int sw = 0; sw < sweeps; ++sw) {
                for (int i = 0; i < N; ++i) {
                    for (int s = 0; s < q; ++s) logit[s] = h[(size_t)i * q + s];
                    for (int e = nbr_ptr[i]; e < nbr_ptr[i + 1]; ++e) {
                        const double *blk = nbr_blk + (size_t)e * q * q;
                        int sj = sig[nbr_idx[e]];
                        for (int s = 0; s < q; ++s) logit[s] += blk[s * q + sj];
                    }
                    double mx = logit[0];
                    for (int s = 1; s < q; ++s)
                        if (logit[s] > mx) mx = logit[s];
                    double acc = 0.0;
                    for (int s = 0; s < q; ++s) {
                        acc += exp(logit[s] - mx);
                        cum[s] = acc;
                    }
                    philox_ctr c = {{(uint32_t)i, (uint32_t)sw, (uint32_t)b, 0u}};
                    double u = u01(philox4x32_10(c, seed, 0u)) * acc;
                    int s = 0;
                    while (s < q - 1 && cum[s] <= u) s++;
                    sig[i] = (int8_t)s;
                }
            }
            for (int i = 0; i < N; ++i) out[(size_t)b * N + i] = sig[i];
        }
        free(sig);
        free(logit);
        free(cum);
    }
    return 0;
}
