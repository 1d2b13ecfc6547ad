/*
 * saim_oracle.c -- plain CPU oracle of the Self-Adaptive Ising Machine (SAIM).
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check of the package entry point and
 * the benchmark's CPU-baseline leg are the only users of this file.  The GPU library shares no
 * code, header, table or constant generator with it, and neither side includes the other.
 *
 * It follows C. Delacour, "Self-Adaptive Ising Machines for Constrained Optimization"
 * (arXiv 2501.04971) step by step, in the paper's order and notation:
 *   - the constrained problem  min f(x) s.t. g(x) = 0                       (Sec. II, Eq. 2)
 *   - penalty energy E = f + P ||g||^2                                     (Sec. II-A, Eq. 3)
 *   - Lagrange function L = E + lambda^T g                                  (Sec. II-B, Eq. 5)
 *   - Algorithm 1: lambda_0 = 0, P = alpha d N, K x {minimise L_k, store feasible x_k,
 *     lambda <- lambda + eta g(x_k)}, return the best stored feasible x  (Sec. III-A, Alg. 1)
 *   - the Ising form of L (Eq. 1) and the p-bit machine I_i = sum_j J_ij m_j + h_i (Eq. 9),
 *     m_i = sign(tanh(beta I_i) + rand(-1,1)) (Eq. 10), updated sequentially spin by spin with a
 *     linear beta schedule from 0 to beta_max; the last sample of each run is x_k (Sec. III-B)
 *   - QKP / MKP with binary slack spins, normalised coefficients, feasibility on the items and
 *     the cost c(x) = -x^T W x / 2 - h^T x                                 (Sec. IV-A, Eq. 12-13;
 *                                                                         Sec. IV-B, Eq. 14)
 *
 * Arithmetic: objective and constraint values in int64 (exact); fields and energies in FP64.
 * The problem scalars sigma_f, sigma_g, P, the inverse temperatures beta_t and the multipliers
 * lambda are FP32 values (rounded once from FP64); every later formula uses those FP32 values
 * widened to FP64.  Build with -ffp-contract=off: the multiplier step is a short FP64 expression
 * whose rounding the GPU path reproduces operation by operation.
 *
 * Readings of points the paper leaves open (each one is also listed in the design notes):
 *   - sign(0) in Eq. 10 is taken as -1, i.e. m_i = +1 iff tanh(beta I_i) + rho > 0 strictly.
 *   - rand(-1,1): rho = (2v+1)/2^24 - 1 with v the top 24 bits of a Philox4x32-10 word; rho is
 *     an odd multiple of 2^-24, never 0 and never +-1.
 *   - beta_t = beta_max * t / (T-1) for sweep t = 0..T-1 (beta_0 = 0; T = 1 gives beta_max).
 *   - every annealing run starts from x = 0 (m = -1); lambda persists across runs.
 *   - spins are visited in index order: items 0..n-1, then the slack bits of constraint 0
 *     (q = 0..Q_0-1), then those of constraint 1, and so on.
 *   - sigma_f = 1/max(|W|,|h|), sigma_g = 1/max(|A|,|b|) over the item coefficients and all
 *     capacities (one scale for all constraints); the multiplier step uses the normalised
 *     constraint sigma_g g, averaged over the C chains of a batch and optionally projected on
 *     lambda >= 0 (C = 1 without projection is Algorithm 1 verbatim).
 *   - d in P = alpha d N: the caller's value when given; otherwise the measured density of the
 *     profit matrix (QKP: nonzero p_ij, i <= j, over n(n+1)/2) or 2/(N+1) without a quadratic
 *     term (MKP, Sec. IV-B), with N the spin count including slack spins (Sec. III-A).
 *   - the stored samples are the last sample of every chain of every run; ties in the final
 *     argmin keep the first achiever in (iteration, chain) order.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------------------------ */
/* Problem extension: binary slack spins (Sec. IV-A, after Eq. 12)                             */
/* ------------------------------------------------------------------------------------------ */

/* Q = floor(log2(b)) + 1 binary slack variables encode 0 <= x_S <= b (Sec. IV-A).  For b >= 1
 * this is the number of binary digits of b. */
/* Threads of the OpenMP loops over chains (timing the oracle on one core or on all). */
OR_API void or_set_threads(int32_t n) { omp_set_num_threads(n > 0 ? n : 1); }
OR_API int32_t or_max_threads(void) { return (int32_t)omp_get_max_threads(); }

OR_API int32_t or_slack_bits(int64_t b) {
    int32_t q = 0;
    if (b <= 0) return 0;
    while (b > 0) {
        q++;
        b >>= 1;
    }
    return q;
}

/* N' = n + sum_k Q_k: the items followed by the slack spins of every constraint. */
OR_API int32_t or_num_spins(int32_t n, int32_t m, const int64_t *b) {
    int32_t N = n;
    for (int32_t k = 0; k < m; k++) N += or_slack_bits(b[k]);
    return N;
}

/* Extended constraint matrix (m x N', row-major): A^T x + x_S = b with x_S = sum_q 2^q x_S^q,
 * so constraint k gets its own Q_k slack columns with coefficients 1, 2, 4, ...  The profits
 * W, h are padded with zeros for the slack spins (Sec. IV-A). */
OR_API void or_extend(int32_t n, int32_t m, const int64_t *A, const int64_t *b, int32_t nprime,
                      int64_t *Aext) {
    memset(Aext, 0, sizeof(int64_t) * (size_t)m * (size_t)nprime);
    int32_t col = n;
    for (int32_t k = 0; k < m; k++) {
        for (int32_t i = 0; i < n; i++) Aext[(size_t)k * nprime + i] = A[(size_t)k * n + i];
        int32_t Q = or_slack_bits(b[k]);
        for (int32_t q = 0; q < Q; q++) Aext[(size_t)k * nprime + col + q] = (int64_t)1 << q;
        col += Q;
    }
}

/* Normalisation and penalty (Sec. IV-A: W, h by max(|W|,|h|) and A, b by max(|A|,|b|), the
 * same for MKP in Sec. IV-B; Sec. III-A: P = alpha d N with N counting the slack spins;
 * Sec. IV-B: d = 2/(N+1) when there is no quadratic profit).  W may be NULL (MKP).
 * out3 = {sigma_f, sigma_g, P} as FP32; *d_used receives the density that entered P. */
OR_API void or_scales(int32_t n, int32_t m, const int64_t *W, const int64_t *h, const int64_t *A,
                      const int64_t *b, int32_t nprime, float alpha, float density, float penalty,
                      float *out3, double *d_used) {
    int64_t mf = 0, mg = 0, nz = 0;
    for (int32_t i = 0; i < n; i++) {
        int64_t v = llabs(h[i]);
        if (v > mf) mf = v;
        if (h[i] != 0) nz++;
        if (W) {
            for (int32_t j = 0; j < n; j++) {
                int64_t w = llabs(W[(size_t)i * n + j]);
                if (w > mf) mf = w;
                if (j > i && W[(size_t)i * n + j] != 0) nz++;
            }
        }
    }
    for (int32_t k = 0; k < m; k++) {
        for (int32_t i = 0; i < n; i++) {
            int64_t v = llabs(A[(size_t)k * n + i]);
            if (v > mg) mg = v;
        }
        int64_t v = llabs(b[k]);
        if (v > mg) mg = v;
    }
    float sf = mf > 0 ? (float)(1.0 / (double)mf) : 1.0f;
    float sg = mg > 0 ? (float)(1.0 / (double)mg) : 1.0f;
    double d;
    if (density >= 0.0f)
        d = (double)density;
    else if (W == NULL)
        d = 2.0 / ((double)nprime + 1.0);
    else
        d = (double)nz / (0.5 * (double)n * (double)(n + 1));
    float P = penalty > 0.0f ? penalty : (float)((double)alpha * d * (double)nprime);
    out3[0] = sf;
    out3[1] = sg;
    out3[2] = P;
    if (d_used) *d_used = d;
}

/* ------------------------------------------------------------------------------------------ */
/* Objective, constraints, feasibility (Sec. IV-A, Eq. 12-13; Sec. IV-B, Eq. 14)               */
/* ------------------------------------------------------------------------------------------ */

/* c(x) = -x^T W x / 2 - h^T x over the n items (W may be NULL: linear MKP objective). */
OR_API int64_t or_cost(int32_t n, const int64_t *W, const int64_t *h, const uint8_t *x) {
    int64_t quad = 0, lin = 0;
    for (int32_t i = 0; i < n; i++) {
        if (!x[i]) continue;
        lin += h[i];
        if (W)
            for (int32_t j = 0; j < n; j++)
                if (x[j]) quad += W[(size_t)i * n + j];
    }
    return -quad / 2 - lin;
}

/* g(x) = A_ext x - b over all N' spins: the equality constraint of the slack-extended problem,
 * g(x) = 0 in Eq. 2. */
OR_API void or_constraints(int32_t m, int32_t nprime, const int64_t *Aext, const int64_t *b,
                           const uint8_t *x, int64_t *g) {
    for (int32_t k = 0; k < m; k++) {
        int64_t s = 0;
        for (int32_t i = 0; i < nprime; i++)
            if (x[i]) s += Aext[(size_t)k * nprime + i];
        g[k] = s - b[k];
    }
}

/* Feasibility check of Sec. IV-A: A^T x <= b on the items only (slack spins ignored). */
OR_API int32_t or_feasible(int32_t n, int32_t m, const int64_t *A, const int64_t *b,
                           const uint8_t *x) {
    for (int32_t k = 0; k < m; k++) {
        int64_t s = 0;
        for (int32_t i = 0; i < n; i++)
            if (x[i]) s += A[(size_t)k * n + i];
        if (s > b[k]) return 0;
    }
    return 1;
}

/* Normalised Lagrange function, Eq. 5 with E of Eq. 3:
 *   L(x) = sigma_f c(x) + P sum_k (sigma_g g_k)^2 + sum_k lambda_k sigma_g g_k. */
OR_API double or_lagrangian(int32_t n, int32_t m, int32_t nprime, const int64_t *W,
                            const int64_t *h, const int64_t *Aext, const int64_t *b,
                            const float *lambda, float sf, float sg, float P, const uint8_t *x) {
    double L = (double)sf * (double)or_cost(n, W, h, x);
    for (int32_t k = 0; k < m; k++) {
        int64_t s = 0;
        for (int32_t i = 0; i < nprime; i++)
            if (x[i]) s += Aext[(size_t)k * nprime + i];
        double gn = (double)sg * (double)(s - b[k]);
        L += (double)P * gn * gn + (double)lambda[k] * gn;
    }
    return L;
}

/* ------------------------------------------------------------------------------------------ */
/* Ising form of L (Eq. 1); J and h change with lambda at every iteration (Sec. III-A)         */
/* ------------------------------------------------------------------------------------------ */

/* Writes the full symmetric N'xN' coupling matrix J (zero diagonal) and the fields hI such that
 * L(x) = H(m) + const for m = 2x - 1, H = -sum_{i<j} J_ij m_i m_j - sum_i h_i m_i (Eq. 1), and
 * returns const.  Derivation: expand L as a QUBO, L = c0 + sum_i q_i x_i + sum_{i<j} R_ij x_i x_j
 * (using x_i^2 = x_i), then substitute x = (1+m)/2:
 *   J_ij = -R_ij/4,  h_i = -q_i/2 - sum_{j!=i} R_ij/4,  const = c0 + sum_i q_i/2 + sum_{i<j} R_ij/4.
 * The QUBO terms are
 *   sigma_f c(x):           R_ij -= sigma_f W_ij,  q_i -= sigma_f h_i
 *   lambda_k sigma_g g_k:   q_i += sigma_g lambda_k a_ki,  c0 -= sigma_g lambda_k b_k
 *   P (sigma_g g_k)^2:      R_ij += 2 P sigma_g^2 a_ki a_kj,  q_i += P sigma_g^2 (a_ki^2 - 2 b_k a_ki),
 *                           c0 += P sigma_g^2 b_k^2. */
OR_API double or_ising(int32_t n, int32_t m, int32_t nprime, const int64_t *W, const int64_t *h,
                       const int64_t *Aext, const int64_t *b, const float *lambda, float sf,
                       float sg, float P, double *J, double *hI) {
    const size_t NN = (size_t)nprime * (size_t)nprime;
    double *R = J; /* the QUBO matrix is built in place, then mapped to J */
    double *q = (double *)calloc((size_t)nprime, sizeof(double));
    const double sfd = sf, sgd = sg, pen = (double)P * (double)sg * (double)sg;
    double c0 = 0.0;
    memset(R, 0, NN * sizeof(double));
    for (int32_t i = 0; i < n; i++) {
        q[i] -= sfd * (double)h[i];
        if (W)
            for (int32_t j = 0; j < n; j++)
                if (j != i) R[(size_t)i * nprime + j] -= sfd * (double)W[(size_t)i * n + j];
    }
    for (int32_t k = 0; k < m; k++) {
        const int64_t *a = Aext + (size_t)k * nprime;
        const double lk = (double)lambda[k], bk = (double)b[k];
        for (int32_t i = 0; i < nprime; i++) {
            if (a[i] == 0) continue;
            const double ai = (double)a[i];
            q[i] += sgd * lk * ai;
            q[i] += pen * (ai * ai - 2.0 * bk * ai);
            for (int32_t j = 0; j < nprime; j++)
                if (j != i && a[j] != 0) R[(size_t)i * nprime + j] += 2.0 * pen * ai * (double)a[j];
        }
        c0 += -sgd * lk * bk + pen * bk * bk;
    }
    double cst = c0;
    for (int32_t i = 0; i < nprime; i++) {
        cst += q[i] / 2.0;
        double rs = 0.0;
        for (int32_t j = 0; j < nprime; j++) {
            if (j == i) continue;
            rs += R[(size_t)i * nprime + j];
            if (j > i) cst += R[(size_t)i * nprime + j] / 4.0;
        }
        hI[i] = -q[i] / 2.0 - rs / 4.0;
    }
    for (size_t e = 0; e < NN; e++) J[e] = -R[e] / 4.0;
    free(q);
    return cst;
}

/* H(m) of Eq. 1 for spins m_i = 2x_i - 1. */
OR_API double or_ising_energy(int32_t nprime, const double *J, const double *hI,
                              const uint8_t *x) {
    double H = 0.0;
    for (int32_t i = 0; i < nprime; i++) {
        const double mi = x[i] ? 1.0 : -1.0;
        H -= hI[i] * mi;
        for (int32_t j = i + 1; j < nprime; j++)
            H -= J[(size_t)i * nprime + j] * mi * (x[j] ? 1.0 : -1.0);
    }
    return H;
}

/* ------------------------------------------------------------------------------------------ */
/* Noise of the p-bit: Philox4x32-10 counter-based generator                                  */
/* ------------------------------------------------------------------------------------------ */

/* Philox4x32 with 10 rounds, as published by Salmon, Moraes, Dror and Shaw ("Parallel random
 * numbers: as easy as 1, 2, 3", SC'11).  One round: the two 32x32->64 products of counter words
 * 0 and 2 with the round multipliers, their high halves xor-ed with the other counter words and
 * the key, a word permutation; between rounds the key advances by the Weyl constants. */
OR_API void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n1 = (uint32_t)p1;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        const uint32_t n3 = (uint32_t)p0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* rand(-1,1) of Eq. 10 from one 32-bit word: rho = (2v+1)/2^24 - 1, v = word >> 8. */
OR_API double or_rand_pm1(uint32_t word) {
    const uint32_t v = word >> 8;
    return ((double)(2u * v + 1u) - 16777216.0) / 16777216.0;
}

/* Noise for (seed, outer iteration k, chain c, sweep t, spin i): Philox4x32-10 with key
 * (low word of seed, high word of seed) and counter (i >> 2, t, c, k); word i & 3 is used. */
OR_API double or_pbit_noise(uint64_t seed, uint32_t iter, uint32_t chain, uint32_t sweep,
                            uint32_t spin) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const uint32_t ctr[4] = {spin >> 2, sweep, chain, iter};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return or_rand_pm1(out[spin & 3u]);
}

/* Linear beta schedule from 0 to beta_max over T sweeps (Sec. III-B), one FP32 value per sweep. */
OR_API float or_beta(float beta_max, int32_t t, int32_t T) {
    if (T <= 1) return beta_max;
    return (float)((double)beta_max * (double)t / (double)(T - 1));
}

/* ------------------------------------------------------------------------------------------ */
/* The p-bit Ising machine (Sec. III-B, Eq. 9-10)                                             */
/* ------------------------------------------------------------------------------------------ */

/* Input of p-bit i, Eq. 9: I_i = sum_j J_ij m_j + h_i. */
static double pbit_input(int32_t nprime, const double *J, const double *hI, const int8_t *mspin,
                         int32_t i) {
    const double *Ji = J + (size_t)i * nprime;
    double I = 0.0;
    for (int32_t j = 0; j < nprime; j++) I += Ji[j] * (double)mspin[j];
    return I + hI[i];
}

/* One sequential Gibbs sweep (Sec. III-B): spins 0..N'-1 in order, each set by Eq. 10,
 * m_i = sign(tanh(beta I_i) + rho), sign(0) = -1. */
static void pbit_sweep(int32_t nprime, const double *J, const double *hI, float beta,
                       uint64_t seed, uint32_t iter, uint32_t chain, uint32_t t, int8_t *mspin) {
    for (int32_t i = 0; i < nprime; i++) {
        const double I = pbit_input(nprime, J, hI, mspin, i);
        const double rho = or_pbit_noise(seed, iter, chain, t, (uint32_t)i);
        mspin[i] = (tanh((double)beta * I) + rho > 0.0) ? 1 : -1;
    }
}

/* Annealing runs (Sec. III-B): chains chain0 .. chain0+nchains-1, each from x = 0 through T
 * sweeps at beta_t; x_out receives the last sample of every chain (nchains x N', 0/1).  If
 * trace is not NULL it receives the state after every sweep (nchains x T x N'). */
OR_API void or_anneal(int32_t nprime, const double *J, const double *hI, float beta_max,
                      int32_t T, uint64_t seed, uint32_t iter, int32_t chain0, int32_t nchains,
                      uint8_t *x_out, uint8_t *trace) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t c = 0; c < nchains; c++) {
        int8_t *ms = (int8_t *)malloc((size_t)nprime);
        for (int32_t i = 0; i < nprime; i++) ms[i] = -1;
        for (int32_t t = 0; t < T; t++) {
            pbit_sweep(nprime, J, hI, or_beta(beta_max, t, T), seed, iter,
                       (uint32_t)(chain0 + c), (uint32_t)t, ms);
            if (trace) {
                uint8_t *tr = trace + ((size_t)c * T + t) * nprime;
                for (int32_t i = 0; i < nprime; i++) tr[i] = ms[i] > 0;
            }
        }
        for (int32_t i = 0; i < nprime; i++) x_out[(size_t)c * nprime + i] = ms[i] > 0;
        free(ms);
    }
}

/* Gibbs sampling at a fixed beta (the Boltzmann law of Eq. 11 is its stationary distribution):
 * nchains independent chains from x = 0, each run for `sweeps` sweeps with outer-iteration index
 * `iter`; the final state of chain c is returned as the integer sum_i x_i 2^i (N' <= 32). */
OR_API void or_gibbs_fixed(int32_t nprime, const double *J, const double *hI, float beta,
                           int32_t sweeps, uint64_t seed, uint32_t iter, int64_t nchains,
                           uint32_t *state_out) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nchains; c++) {
        int8_t ms[32];
        for (int32_t i = 0; i < nprime; i++) ms[i] = -1;
        for (int32_t t = 0; t < sweeps; t++)
            pbit_sweep(nprime, J, hI, beta, seed, iter, (uint32_t)c, (uint32_t)t, ms);
        uint32_t s = 0;
        for (int32_t i = 0; i < nprime; i++)
            if (ms[i] > 0) s |= 1u << i;
        state_out[c] = s;
    }
}

/* Teacher-forced replay of one recorded sweep.  Starting from the recorded state x0 (0/1), each
 * spin i in order gets the oracle's decision from the current state, which is compared with the
 * recorded decision x1[i]; the state then continues from x1[i].  Returns the number of
 * disagreements; for each of the first max_out disagreements, spin_out receives the spin index and
 * margin_out the value tanh(beta I_i) + rho the oracle saw (its sign is the oracle's decision). */
OR_API int32_t or_replay_sweep(int32_t nprime, const double *J, const double *hI, float beta,
                               uint64_t seed, uint32_t iter, uint32_t chain, uint32_t t,
                               const uint8_t *x0, const uint8_t *x1, int32_t *spin_out,
                               double *margin_out, int32_t max_out) {
    int8_t *ms = (int8_t *)malloc((size_t)nprime);
    int32_t bad = 0;
    for (int32_t i = 0; i < nprime; i++) ms[i] = x0[i] ? 1 : -1;
    for (int32_t i = 0; i < nprime; i++) {
        const double I = pbit_input(nprime, J, hI, ms, i);
        const double rho = or_pbit_noise(seed, iter, chain, t, (uint32_t)i);
        const double v = tanh((double)beta * I) + rho;
        const int mine = v > 0.0;
        if (mine != (int)(x1[i] != 0)) {
            if (bad < max_out) {
                spin_out[bad] = i;
                margin_out[bad] = v;
            }
            bad++;
        }
        ms[i] = x1[i] ? 1 : -1;
    }
    free(ms);
    return bad;
}

/* ------------------------------------------------------------------------------------------ */
/* Algorithm 1: multiplier update, the outer loop, and the final selection                    */
/* ------------------------------------------------------------------------------------------ */

/* The multiplier step with a step-size rule.  Sec. III-A ascends the dual along the
 * subgradient g(x) and notes that the surrogate-gradient method converges with approximate
 * minimisers too; that method lets the step size shrink and the direction be a combination of
 * recent subgradients.  The two variants here (not in the paper; definitions, not readings):
 *   eta_it = eta / (1 + decay it)        (eta_sqrt = 0)
 *   eta_it = eta / sqrt(1 + decay it)    (eta_sqrt = 1), it = the outer-iteration index;
 *   d = mu avg + (1 - mu) mean, stored back into avg (an exponentially weighted average of
 *   the batch-mean subgradients, avg = 0 before the first step); mu = 0 gives d = mean.
 * lambda_k <- lambda_k + eta_it sigma_g d_k, projected on lambda >= 0 if asked, rounded to FP32.
 * FP64, evaluated in this order without fused operations: mean = S/C; d; den = 1 + decay*it
 * (its square root if eta_sqrt); eta_it = eta/den (eta itself when decay = 0);
 * step = eta_it*(sigma_g*d); l = lambda + step.  avg may be NULL when mu = 0. */
OR_API void or_lambda_update_rule(int32_t m, const int64_t *gsum, int64_t C, double eta,
                                  int32_t project, float sg, uint32_t it, double decay,
                                  int32_t eta_sqrt, double mu, double *avg, float *lambda) {
    double eta_it = eta;
    if (decay != 0.0) {
        double den = 1.0 + decay * (double)it;
        if (eta_sqrt) den = sqrt(den);
        eta_it = eta / den;
    }
    for (int32_t k = 0; k < m; k++) {
        const double mean = (double)gsum[k] / (double)C;
        double d = mean;
        if (mu != 0.0) {
            d = mu * avg[k] + (1.0 - mu) * mean;
            avg[k] = d;
        }
        const double step = eta_it * ((double)sg * d);
        double l = (double)lambda[k] + step;
        if (project && l < 0.0) l = 0.0;
        lambda[k] = (float)l;
    }
}

/* lambda_{k+1} = lambda_k + eta g(x_k) (Algorithm 1) with g in normalised units (sigma_g g),
 * gsum[k] = sum over the C chains of g_k (int64, exact), mean over chains, optional projection
 * on lambda >= 0.  FP64 evaluation order: mean = S/C; step = eta*(sigma_g*mean); l = lambda+step;
 * the result is rounded to FP32.  (The rule above with a constant step and no averaging.) */
OR_API void or_lambda_update(int32_t m, const int64_t *gsum, int64_t C, double eta,
                             int32_t project, float sg, float *lambda) {
    or_lambda_update_rule(m, gsum, C, eta, project, sg, 0u, 0.0, 0, 0.0, NULL, lambda);
}

/* Best feasible state among the sweep-end states of C annealing runs.  The paper checks every
 * measured sample for feasibility and stores the feasible ones (Sec. IV-A; Algorithm 1's "store
 * feasible"); a run's last state is its measured sample.  This option measures the state at the
 * end of every sweep t = 0..T-1 instead: trace[c][t] (N' bytes each).  For chain c: the states
 * feasible under capacities b_check (items only, A x <= b_check), the one of least cost c(x)
 * (Sec. IV-A), the earliest sweep on ties.  Outputs per chain: best_cost (INT64_MAX if none),
 * best_x (N' bytes, zeros if none), best_sweep (-1 if none), nfeas (feasible sweep-end states;
 * any output may be NULL). */
OR_API void or_run_best(int32_t n, int32_t m, int32_t nprime, const int64_t *W, const int64_t *h,
                        const int64_t *A, const int64_t *b_check, int32_t C, int32_t T,
                        const uint8_t *trace, int64_t *best_cost, uint8_t *best_x,
                        int32_t *best_sweep, int32_t *nfeas) {
    for (int32_t c = 0; c < C; c++) {
        int64_t bc = INT64_MAX;
        int32_t bt = -1, nf = 0;
        for (int32_t t = 0; t < T; t++) {
            const uint8_t *x = trace + ((size_t)c * T + t) * nprime;
            if (!or_feasible(n, m, A, b_check, x)) continue;
            nf++;
            const int64_t cost = or_cost(n, W, h, x);
            if (cost < bc) {
                bc = cost;
                bt = t;
            }
        }
        if (best_cost) best_cost[c] = bc;
        if (best_sweep) best_sweep[c] = bt;
        if (nfeas) nfeas[c] = nf;
        if (best_x) {
            uint8_t *bx = best_x + (size_t)c * nprime;
            if (bt >= 0)
                memcpy(bx, trace + ((size_t)c * T + bt) * nprime, (size_t)nprime);
            else
                memset(bx, 0, (size_t)nprime);
        }
    }
}

/* Algorithm 1 for K iterations k = iter0 .. iter0+K-1 on one instance.  Per iteration: J, h of
 * L_k from lambda_k; C annealing runs (the Ising machine minimising L_k); every chain's last
 * sample is checked, feasible ones are stored (only the best is kept: min cost, first achiever
 * in (k, chain) order); lambda takes the batch-mean subgradient step on the last samples.
 * b_check (NULL: b) are the capacities that feasibility is checked against: the problem L is
 * built from b, and b_check > b is the capacity tightening B' < B of Sec. IV-B (b holding B').
 * run_best = 1: the sample stored from a chain is its best feasible sweep-end state
 * (or_run_best) instead of its last state; lambda still steps on the last states.
 * eta_decay, eta_sqrt, mu: the step-size rule of or_lambda_update_rule (0, 0, 0: Algorithm 1's
 * constant step), with the outer-iteration index kk and the average starting at 0.
 * Outputs: *best_cost (INT64_MAX if nothing feasible), best_x (N' bytes), best_iter/best_chain,
 * lambda_trace (K x m: lambda after each update, may be NULL), *feasible_count (stored feasible
 * samples), and optionally every last sample's cost (K x C) and constraint values (K x C x m). */
OR_API void or_solve(int32_t n, int32_t m, const int64_t *W, const int64_t *h, const int64_t *A,
                     const int64_t *b, const int64_t *b_check, float alpha, float density,
                     float penalty, int32_t K, int32_t C, int32_t T, float beta_max, double eta,
                     uint64_t seed, uint32_t iter0, int32_t project, int32_t run_best,
                     double eta_decay, int32_t eta_sqrt, double mu,
                     const float *lambda0, int64_t *best_cost, uint8_t *best_x,
                     int32_t *best_iter, int32_t *best_chain, float *lambda_trace,
                     int64_t *feasible_count, int64_t *cost_out, int64_t *g_out) {
    if (!b_check) b_check = b;
    const int32_t nprime = or_num_spins(n, m, b);
    int64_t *Aext = (int64_t *)malloc(sizeof(int64_t) * (size_t)m * nprime);
    or_extend(n, m, A, b, nprime, Aext);
    float sc[3];
    or_scales(n, m, W, h, A, b, nprime, alpha, density, penalty, sc, NULL);
    double *J = (double *)malloc(sizeof(double) * (size_t)nprime * nprime);
    double *hI = (double *)malloc(sizeof(double) * (size_t)nprime);
    uint8_t *xs = (uint8_t *)malloc((size_t)C * nprime);
    float *lambda = (float *)malloc(sizeof(float) * (size_t)(m > 0 ? m : 1));
    int64_t *g = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    int64_t *gsum = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    double *avg = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    uint8_t *trace = run_best ? (uint8_t *)malloc((size_t)C * T * nprime) : NULL;
    int64_t *rcost = run_best ? (int64_t *)malloc(sizeof(int64_t) * (size_t)C) : NULL;
    uint8_t *rx = run_best ? (uint8_t *)malloc((size_t)C * nprime) : NULL;
    for (int32_t k = 0; k < m; k++) lambda[k] = lambda0 ? lambda0[k] : 0.0f;
    *best_cost = INT64_MAX;
    *best_iter = -1;
    *best_chain = -1;
    *feasible_count = 0;
    for (int32_t it = 0; it < K; it++) {
        const uint32_t kk = iter0 + (uint32_t)it;
        or_ising(n, m, nprime, W, h, Aext, b, lambda, sc[0], sc[1], sc[2], J, hI);
        or_anneal(nprime, J, hI, beta_max, T, seed, kk, 0, C, xs, trace);
        if (run_best) or_run_best(n, m, nprime, W, h, A, b_check, C, T, trace, rcost, rx, NULL, NULL);
        for (int32_t k = 0; k < m; k++) gsum[k] = 0;
        for (int32_t c = 0; c < C; c++) {
            const uint8_t *x = xs + (size_t)c * nprime;
            const int64_t cost = or_cost(n, W, h, x);
            or_constraints(m, nprime, Aext, b, x, g);
            for (int32_t k = 0; k < m; k++) gsum[k] += g[k];
            if (cost_out) cost_out[(size_t)it * C + c] = cost;
            if (g_out)
                for (int32_t k = 0; k < m; k++) g_out[((size_t)it * C + c) * m + k] = g[k];
            /* the sample stored from this chain: its last state, or its best sweep-end state */
            const int stored = run_best ? rcost[c] != INT64_MAX : or_feasible(n, m, A, b_check, x);
            const int64_t scost = run_best ? rcost[c] : cost;
            const uint8_t *sx = run_best ? rx + (size_t)c * nprime : x;
            if (stored) {
                (*feasible_count)++;
                if (scost < *best_cost) {
                    *best_cost = scost;
                    *best_iter = (int32_t)kk;
                    *best_chain = c;
                    memcpy(best_x, sx, (size_t)nprime);
                }
            }
        }
        or_lambda_update_rule(m, gsum, C, eta, project, sc[1], kk, eta_decay, eta_sqrt, mu, avg,
                              lambda);
        if (lambda_trace)
            for (int32_t k = 0; k < m; k++) lambda_trace[(size_t)it * m + k] = lambda[k];
    }
    free(Aext);
    free(J);
    free(hI);
    free(xs);
    free(lambda);
    free(g);
    free(gsum);
    free(avg);
    free(trace);
    free(rcost);
    free(rx);
}

/* ------------------------------------------------------------------------------------------ */
/* Exhaustive references for small instances                                                  */
/* ------------------------------------------------------------------------------------------ */

/* L(x) of Eq. 5 for every state x of N' <= 24 spins (x_i = bit i of the index). */
OR_API void or_enumerate_lagrangian(int32_t n, int32_t m, int32_t nprime, const int64_t *W,
                                    const int64_t *h, const int64_t *Aext, const int64_t *b,
                                    const float *lambda, float sf, float sg, float P,
                                    double *L_out) {
    const int64_t S = (int64_t)1 << nprime;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < S; s++) {
        uint8_t x[32];
        for (int32_t i = 0; i < nprime; i++) x[i] = (uint8_t)((s >> i) & 1);
        L_out[s] = or_lagrangian(n, m, nprime, W, h, Aext, b, lambda, sf, sg, P, x);
    }
}

/* Constrained optimum OPT of Eq. 2 by enumeration of the n <= 24 items: min c(x) s.t. A x <= b.
 * Returns INT64_MAX if no state is feasible; x_best receives the first minimiser (lowest index). */
OR_API int64_t or_brute_force_opt(int32_t n, int32_t m, const int64_t *W, const int64_t *h,
                                  const int64_t *A, const int64_t *b, uint8_t *x_best) {
    const int64_t S = (int64_t)1 << n;
    int64_t best = INT64_MAX, arg = -1;
    uint8_t x[32];
    for (int64_t s = 0; s < S; s++) {
        for (int32_t i = 0; i < n; i++) x[i] = (uint8_t)((s >> i) & 1);
        if (!or_feasible(n, m, A, b, x)) continue;
        const int64_t c = or_cost(n, W, h, x);
        if (c < best) {
            best = c;
            arg = s;
        }
    }
    if (arg >= 0 && x_best)
        for (int32_t i = 0; i < n; i++) x_best[i] = (uint8_t)((arg >> i) & 1);
    return best;
}
