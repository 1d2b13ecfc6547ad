/*
 * mlp_oracle.c -- plain CPU oracle of the learned multiplier warm start.
 *
 * TEST INFRASTRUCTURE ONLY, like saim_oracle.c: the tests, the smoke check and the benchmark's
 * CPU leg are its only users, and it shares no code with the GPU library.
 *
 * The paper has no learned part; this follows its definition as a plain multilayer perceptron
 * (in the notation of a textbook two-hidden-layer ReLU network) written out in FP64:
 *
 *   features of constraint k (built on Sec. IV-A's normalised coefficients):
 *     f0 = min(1, b_k / sum_i a_ki)      (1 when the row sum is 0)
 *     f1 = sigma_g * mean_i a_ki,  f2 = sigma_g * std_i a_ki        (items i < n, population std)
 *     f3 = sigma_f * mean p,       f4 = sigma_f * std p   over the nonzero profits
 *                                       {h_i} and {W_ij, i < j}
 *     f5 = n / 1000,               f6 = d  (the density that entered P = alpha d N, Sec. III-A)
 *   network, x'_f = (x_f - mu_f) / sd_f for f < 7, x'_7 = 1 (the bias input):
 *     z1 = W1 x'            (W1: 128 x 16, column 7 = b1, columns 8..15 zero)
 *     h1 = relu(z1), h1_128 = 1
 *     z2 = W2 h1            (W2: 128 x 144, column 128 = b2, columns 129..143 zero)
 *     h2 = relu(z2)
 *     u  = w3 . h2 + b3,    lambda_k = y_mu + y_sd * u
 *   loss on normalised targets t' = (t - y_mu) / y_sd:  (1/B) sum_r (u_r - t'_r)^2, its
 *   gradient by the chain rule (relu'(0) = 0), and one Adam step (Kingma & Ba, Algorithm 1):
 *     m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, theta -= lr (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps).
 *
 * Flat parameter vector (PARAMS = 20612): W1 at 0 (2048), W2 at 2048 (18432), w3 at 20480
 * (128), b3 at 20608, three unused entries.  norm[16] = {mu[0..6], sd[0..6], y_mu, y_sd}.
 *
 * Precision modes (flags): OR_MLP_BF16 rounds what a BF16 tensor-core implementation feeds its
 * products -- every weight (biases included), x', h1, dz2 and dz1 -- to BF16 (round to nearest
 * even), and keeps everything else in FP64.  OR_MLP_ABS replaces every weight, activation and
 * gradient by its magnitude and every ReLU mask by 1: the result bounds the magnitude of any
 * perturbation carried through the same sums, which the tests turn into tolerances.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define OR_API __attribute__((visibility("default")))

enum { H = 128, NF = 7, K1 = 16, K2 = 144, OFF_W1 = 0, OFF_W2 = 2048, OFF_W3 = 20480,
       OFF_B3 = 20608, PARAMS = 20612 };
enum { OR_MLP_BF16 = 1, OR_MLP_ABS = 2 };

/* Round an FP32 value to BF16 (round to nearest, ties to even); NaN is not produced here. */
OR_API float or_bf16_round(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    u &= 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return f;
}

static double q(double v, int flags) {
    if (flags & OR_MLP_ABS) return fabs(v);
    if (flags & OR_MLP_BF16) return (double)or_bf16_round((float)v);
    return v;
}
static double relu(double v, int flags) { return (flags & OR_MLP_ABS) ? v : (v > 0.0 ? v : 0.0); }
static double mask(double z, int flags) { return (flags & OR_MLP_ABS) ? 1.0 : (z > 0.0 ? 1.0 : 0.0); }

extern void or_scales(int32_t n, int32_t m, const int64_t *W, const int64_t *h, const int64_t *A,
                      const int64_t *b, int32_t nprime, float alpha, float density, float penalty,
                      float *out3, double *d_used);
extern int32_t or_num_spins(int32_t n, int32_t m, const int64_t *b);

/* Per-constraint features (rows m x 8, column 7 zero) of one instance, as listed above. */
OR_API void or_features(int32_t n, int32_t m, const int64_t *W, const int64_t *h, const int64_t *A,
                        const int64_t *b, float alpha, float density, float penalty, float *out) {
    float sc[3];
    double d = 0.0;
    const int32_t nprime = or_num_spins(n, m, b);
    or_scales(n, m, W, h, A, b, nprime, alpha, density, penalty, sc, &d);
    const double sf = sc[0], sg = sc[1];
    /* profits: nonzero h_i and nonzero W_ij above the diagonal */
    double ps = 0.0, pss = 0.0, pc = 0.0;
    for (int i = 0; i < n; ++i) {
        if (h[i] != 0) {
            ps += (double)h[i];
            pss += (double)h[i] * (double)h[i];
            pc += 1.0;
        }
        if (W)
            for (int j = i + 1; j < n; ++j) {
                const double w = (double)W[(size_t)i * n + j];
                if (w != 0.0) {
                    ps += w;
                    pss += w * w;
                    pc += 1.0;
                }
            }
    }
    const double pmean = pc > 0 ? ps / pc : 0.0;
    const double pvar = pc > 0 ? pss / pc - pmean * pmean : 0.0;
    for (int k = 0; k < m; ++k) {
        double s = 0.0, ss = 0.0;
        for (int i = 0; i < n; ++i) {
            const double a = (double)A[(size_t)k * n + i];
            s += a;
            ss += a * a;
        }
        const double mean = s / n, var = ss / n - mean * mean;
        float *o = out + (size_t)k * 8;
        o[0] = (float)(s > 0 ? fmin(1.0, (double)b[k] / s) : 1.0);
        o[1] = (float)(sg * mean);
        o[2] = (float)(sg * sqrt(var > 0 ? var : 0.0));
        o[3] = (float)(sf * pmean);
        o[4] = (float)(sf * sqrt(pvar > 0 ? pvar : 0.0));
        o[5] = (float)(n / 1000.0);
        o[6] = (float)d;
        o[7] = 0.0f;
    }
}

/* Forward pass of one row; fills x' (16), z1, h1 (144 incl. the bias input), z2, h2 and returns
 * the normalised output u. */
static double forward_row(const double *p, const double *norm, const float *x, int flags,
                          double *xp, double *z1, double *h1, double *z2, double *h2) {
    for (int f = 0; f < K1; ++f) {
        double v = 0.0;
        if (f < NF) v = ((double)x[f] - norm[f]) / norm[NF + f];
        else if (f == NF) v = 1.0;
        xp[f] = q(v, flags);
    }
    for (int o = 0; o < H; ++o) {
        double s = 0.0;
        for (int k = 0; k < K1; ++k) s += q(p[OFF_W1 + o * K1 + k], flags) * xp[k];
        z1[o] = s;
        h1[o] = q(relu(s, flags), flags);
    }
    for (int k = H; k < K2; ++k) h1[k] = k == H ? 1.0 : 0.0;
    double u = q(p[OFF_B3], flags);
    for (int o = 0; o < H; ++o) {
        double s = 0.0;
        for (int k = 0; k < K2; ++k) s += q(p[OFF_W2 + o * K2 + k], flags) * h1[k];
        z2[o] = s;
        h2[o] = relu(s, flags);
        u += q(p[OFF_W3 + o], flags) * h2[o];
    }
    return u;
}

static void widen(const float *src, double *dst, int n) {
    for (int i = 0; i < n; ++i) dst[i] = (double)src[i];
}

/* lambda = y_mu + y_sd * u for every row (rows x 8 features). */
OR_API void or_mlp_forward(const float *params, const float *norm, const float *X, int32_t rows,
                           int32_t flags, double *y) {
    static __thread double p[PARAMS];
    double nm[16], xp[K1], z1[H], h1[K2], z2[H], h2[H];
    widen(params, p, PARAMS);
    widen(norm, nm, 16);
    for (int r = 0; r < rows; ++r) {
        const double u = forward_row(p, nm, X + (size_t)r * 8, flags, xp, z1, h1, z2, h2);
        y[r] = (flags & OR_MLP_ABS) ? fabs(nm[15]) * u + fabs(nm[14]) : nm[14] + nm[15] * u;
    }
}

/* Mean squared error over the rows (normalised units) and its gradient w.r.t. the flat
 * parameter vector (PARAMS doubles, padding columns left zero).  Returns the loss. */
OR_API double or_mlp_grad(const float *params, const float *norm, const float *X, const float *t,
                          int32_t rows, int32_t flags, double *grad) {
    static __thread double p[PARAMS];
    double nm[16], xp[K1], z1[H], h1[K2], z2[H], h2[H], dz2[H], dz1[H];
    widen(params, p, PARAMS);
    widen(norm, nm, 16);
    memset(grad, 0, sizeof(double) * PARAMS);
    double loss = 0.0;
    for (int r = 0; r < rows; ++r) {
        const double u = forward_row(p, nm, X + (size_t)r * 8, flags, xp, z1, h1, z2, h2);
        const double tn = ((double)t[r] - nm[14]) / nm[15];
        const double e = (flags & OR_MLP_ABS) ? fabs(u) + fabs(tn) : u - tn;
        loss += e * e;
        const double du = 2.0 * e / rows;
        grad[OFF_B3] += du;
        for (int o = 0; o < H; ++o) {
            grad[OFF_W3 + o] += du * h2[o];
            dz2[o] = q(du * q(p[OFF_W3 + o], flags) * mask(z2[o], flags), flags);
        }
        for (int o = 0; o < H; ++o)
            for (int k = 0; k <= H; ++k) grad[OFF_W2 + o * K2 + k] += dz2[o] * h1[k];
        for (int k = 0; k < H; ++k) {
            double s = 0.0;
            for (int o = 0; o < H; ++o) s += dz2[o] * q(p[OFF_W2 + o * K2 + k], flags);
            dz1[k] = q(s * mask(z1[k], flags), flags);
        }
        for (int o = 0; o < H; ++o)
            for (int k = 0; k <= NF; ++k) grad[OFF_W1 + o * K1 + k] += dz1[o] * xp[k];
    }
    return loss / rows;
}

/* One Adam step (Kingma & Ba, Algorithm 1) at step number t >= 1, in place. */
OR_API void or_adam_step(int32_t n, double *theta, double *mom, double *vel, const double *g,
                         int32_t t, double lr, double b1, double b2, double eps) {
    const double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int i = 0; i < n; ++i) {
        mom[i] = b1 * mom[i] + (1.0 - b1) * g[i];
        vel[i] = b2 * vel[i] + (1.0 - b2) * g[i] * g[i];
        theta[i] -= lr * (mom[i] / c1) / (sqrt(vel[i] / c2) + eps);
    }
}
