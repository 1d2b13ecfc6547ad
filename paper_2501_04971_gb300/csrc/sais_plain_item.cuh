// sais_plain_item.cuh -- the plain per-spin p-bit sampler (Sec. III-B, Eq. 9-10) as a device
// function over one work item; its own kernel is in sais_plain.cu, and the persistent ragged
// kernel (sais_ragged.cu) calls it for linear-objective instances.
//
// Layout.  One thread owns one chain; a work item is `cpb` chains of one instance.
// The objective part of the local field, F_i = h_i + sum_j W_ij x_j (an exact integer held in
// FP32), lives in shared memory chain-minor, F[i][chain], so a warp touching spin i reads and
// writes 32 consecutive words.  The bit-packed state sits beside it.  Per chain the constraint
// values g_k = (A_ext x - b)_k are int32 registers, and c_k = sigma_g lambda_k + 2 P sigma_g^2 g_k
// (FP32) is refreshed whenever g_k changes.
//
// One update of spin i (sequential, i = 0..N'-1, Sec. III-B):
//   2 I_i = sigma_f F_i - sum_k a_ki c_k - (1 - 2 x_i) D_i,  D_i = P sigma_g^2 sum_k a_ki^2,
// which is -dL_i with dL_i = L(x_i = 1) - L(x_i = 0) of Eq. 5 (the p-bit input of Eq. 9 for
// the Ising form of L).  The decision follows sais_device.cuh.  On a flip the constraint values
// change by a_ki and, if any chain of the warp flipped, the warp adds W[i,:] * delta to its
// chains' F columns (rank-1 update, W row broadcast from L1/L2).  The constraint values are
// FP32 (exact integers below 2^24).  After the items, each constraint's slack spins run in a loop
// of their own: a slack spin has a single nonzero coefficient, so its field and its flip touch
// one constraint.
//
// Error bound of the FP32 field (u = 2^-24): t0 = fl(sigma_f F_i) carries u|sigma_f F_i|; each
// c_k carries at most 3.02 u M_k with M_k = |2 P sigma_g^2 g_k| + |sigma_g lambda_k|; the chain
// of m + 1 fused multiply-adds adds gamma_{m+1} times the sum of the magnitudes; D_i carries
// 1.01 u D_i; the final product by beta/2 one more u.  Altogether
//   |z - beta I_i| <= (beta/2) (m + 6.2) u (|sigma_f F_i| + sum_k a_ki M_k + D_i),
// and sum_k a_ki M_k <= (sum_k a_ki) max_k M_k.  field_err_factor() uses m + 12 with a margin.
#pragma once

#include <climits>
#include <type_traits>

#include "sais_device.cuh"

namespace sais {
namespace {

// One work item: chains grp cpb .. grp cpb + cpb - 1 of instance j, one per thread (thread tid
// of the item's cpb), dynamic shared memory sized by plain_smem_bytes for cpb chains (declared
// here, not passed as a pointer, so that every access stays a shared-memory access).  kF16: the
// objective field F is held as int16 (the launch guarantees |F_i| <= |h_i| + sum_j |W_ij| <=
// 32767 for every state, so every value it takes is exact), half the shared memory of FP32 and
// so twice the chains per SM; the arithmetic of the field is the same FP32 on the same values.
template <int MC, bool kF16 = false>
__device__ __forceinline__ void plain_item(const SampleArgs &a, int j, int grp, int cpb, int tid) {
    using FT = typename std::conditional<kF16, int16_t, float>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (!SAIS_DCHECK(a.status, j >= 0 && j < a.count && grp >= 0 && grp * cpb < a.chains))
        return;
    const InstDev *__restrict__ ip = a.inst + j;
    const int n = ip->n, m = ip->m, nprime = ip->nprime, npad = ip->npad, words = ip->words;
    const int m4 = ip->m4;
    const bool has_w = ip->has_w != 0;
    const float sf = ip->sigma_f, sg = ip->sigma_g, kappa = ip->kappa;
    const double psg2 = ip->psg2;
    const int16_t *__restrict__ W = ip->W;
    const float *__restrict__ hF = ip->hF;
    const float *__restrict__ acf = ip->acf;
    const float *__restrict__ Dv = ip->D;
    const float *__restrict__ asum = ip->asum;

    const int chain = grp * cpb + tid;
    const bool valid = chain < (a.inst_chains ? a.inst_chains[j] : a.chains);
    const uint32_t iter = a.iter_dev ? *a.iter_dev : a.iter;
    const uint64_t seed = a.seed + (uint64_t)j;
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);

    FT *Fs = reinterpret_cast<FT *>(smem_raw);
    const size_t fbytes = has_w ? (size_t)npad * cpb * sizeof(FT) : 0;
    uint32_t *xs = reinterpret_cast<uint32_t *>(smem_raw + fbytes);
    // Debug builds: this item's shared memory within the launch's (uniform over the CTA).
    if (!SAIS_DCHECK(a.status, fbytes + (size_t)words * cpb * 4 <= dynamic_smem_bytes()))
        return;

    const float *lam = a.lambda + (size_t)j * a.m_stride;
    // Constraint values g_k as FP32 (exact integers: |g| < 2^24, checked at creation) and
    // c_k = 2 P sigma_g^2 g_k + sigma_g lambda_k.
    float gf[MC], c[MC], cA[MC];
    float Mmax = 0.f;
#pragma unroll
    for (int k = 0; k < MC; ++k) {
        if (k < m) {
            cA[k] = __double2float_rn((double)sg * (double)lam[k]);
            gf[k] = (float)(-ip->b[k]);
            c[k] = fmaf(kappa, gf[k], cA[k]);
            Mmax = fmaxf(Mmax, fmaf(fabsf(kappa), fabsf(gf[k]), fabsf(cA[k])));
        } else {
            cA[k] = 0.f;
            gf[k] = 0.f;
            c[k] = 0.f;
        }
    }
    if (has_w)
        for (int i = 0; i < npad; ++i) Fs[i * cpb + tid] = (FT)hF[i];
    for (int w = 0; w < words; ++w) xs[w * cpb + tid] = 0u;
    const float errk = field_err_factor(m);
    // Best feasible sweep-end state of the run (when a.run_cost is set): the cost of the current
    // state follows every flip, c(x') - c(x) = -d F_i (F_i = h_i + sum_j W_ij x_j, W_ii = 0).
    const bool track = a.run_cost != nullptr;
    long long ccur = 0, rbest = LLONG_MAX;
    int rsweep = -1, rnf = 0;

    for (int t = 0; t < a.sweeps; ++t) {
        const float beta = beta_of_sweep(a.beta_max, t, a.sweeps);
        const float hb = 0.5f * beta;
        const float ez = hb * errk;
        uint32_t xw = 0u;
        uint4 rw = make_uint4(0u, 0u, 0u, 0u);   // noise words of spins 4 (i/4) .. 4 (i/4) + 3
        // Items, spins 0..n-1: objective field and every constraint.
        for (int i0 = 0; i0 < n; i0 += 4) {
            rw = philox4x32_10(
                make_uint4((uint32_t)(i0 >> 2), (uint32_t)t, (uint32_t)chain, iter), key0, key1);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + q;
                if (i >= n) break;
                if ((i & 31) == 0) xw = xs[(i >> 5) * cpb + tid];
                const float theta = theta_of_word(word_of(rw, q));
                const float Fi = has_w ? (float)Fs[i * cpb + tid] : __ldg(hF + i);
                const int xi = (xw >> (i & 31)) & 1;
                // Row i of A_ext as FP32, four coefficients per load.
                float akf[MC];
                if constexpr (MC >= 4) {
                    const float4 *ap = reinterpret_cast<const float4 *>(acf + (size_t)i * m4);
#pragma unroll
                    for (int k4 = 0; k4 < MC / 4; ++k4) {
                        const float4 v = 4 * k4 < m ? __ldg(ap + k4) : make_float4(0.f, 0.f, 0.f, 0.f);
                        akf[4 * k4] = v.x;
                        akf[4 * k4 + 1] = v.y;
                        akf[4 * k4 + 2] = v.z;
                        akf[4 * k4 + 3] = v.w;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < MC; ++k) akf[k] = k < m ? __ldg(acf + (size_t)i * m4 + k) : 0.f;
                }
                float acc = sf * Fi;
                const float tabs = fabsf(acc);
                if constexpr (MC >= 16) {
                    // Four independent partial sums instead of one chain of m fused products
                    // (the bound gamma_{m+1} sum|terms| holds for any order of the additions);
                    // measured faster from m = 30 on, slower at m = 5.
                    float p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
                    for (int k = 0; k < MC; ++k) {
                        float &pk = (k & 3) == 0 ? acc : ((k & 3) == 1 ? p1 : ((k & 3) == 2 ? p2 : p3));
                        pk = fmaf(-akf[k], c[k], pk);
                    }
                    acc = (acc + p1) + (p2 + p3);
                } else {
#pragma unroll
                    for (int k = 0; k < MC; ++k) acc = fmaf(-akf[k], c[k], acc);
                }
                const float Di = __ldg(Dv + i);
                acc = fmaf(xi ? 1.f : -1.f, Di, acc);
                const float z = hb * acc;
                const float y = z + theta;
                const float bound =
                    ez * (tabs + __ldg(asum + i) * Mmax + Di) + kThetaRelErr * fabsf(theta) + kThetaAbsErr;
                int xn;
                if (fabsf(y) > bound) {
                    xn = y > 0.f;
                } else {
                    int32_t ak[MC], g[MC];
#pragma unroll
                    for (int k = 0; k < MC; ++k) {
                        ak[k] = (int32_t)akf[k];
                        g[k] = (int32_t)gf[k];
                    }
                    xn = decide_exact<MC>(Fi, xi, ak, g, lam, m, sf, sg, psg2, beta,
                                          rho_of_word(word_of(rw, q)));
                }
                const int d = xn - xi;
                if (d != 0) {
                    const float df = (float)d;
                    xw ^= 1u << (i & 31);
                    ccur -= (long long)(d * __float2int_rz(Fi));   // |F| < 2^24: exact
                    Mmax = 0.f;
#pragma unroll
                    for (int k = 0; k < MC; ++k) {
                        if (k < m) {
                            gf[k] = fmaf(akf[k], df, gf[k]);   // exact integers
                            c[k] = fmaf(kappa, gf[k], cA[k]);
                            Mmax = fmaxf(Mmax, fmaf(fabsf(kappa), fabsf(gf[k]), fabsf(cA[k])));
                        }
                    }
                }
                if (has_w && __any_sync(0xffffffffu, d != 0)) {
                    const float df = (float)d;
                    const int4 *Wi = reinterpret_cast<const int4 *>(W + (size_t)i * npad);
                    FT *Fc = Fs + tid;
                    for (int j8 = 0; j8 < (npad >> 3); ++j8) {
                        const int4 v = __ldg(Wi + j8);
                        const uint32_t u[4] = {(uint32_t)v.x, (uint32_t)v.y, (uint32_t)v.z,
                                               (uint32_t)v.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int r = (j8 * 8 + 2 * e) * cpb;
                            if constexpr (kF16) {   // integer update, exact in int16
                                const int wlo = (int16_t)(u[e] & 0xffffu);
                                const int whi = (int16_t)(u[e] >> 16);
                                Fc[r] = (int16_t)(Fc[r] + d * wlo);
                                Fc[r + cpb] = (int16_t)(Fc[r + cpb] + d * whi);
                            } else {
                                const float wlo = (float)(int16_t)(u[e] & 0xffffu);
                                const float whi = (float)(int16_t)(u[e] >> 16);
                                Fc[r] = fmaf(df, wlo, Fc[r]);
                                Fc[r + cpb] = fmaf(df, whi, Fc[r + cpb]);
                            }
                        }
                    }
                }
                if ((i & 31) == 31 || i == nprime - 1) xs[(i >> 5) * cpb + tid] = xw;
            }
        }
        // Slack spins of constraint k: spins o_k .. o_{k+1} - 1, bit q with coefficient 2^q in
        // row k of A_ext only (Sec. IV-A).  No pair values and h = 0, so F_i = 0: the field is
        // 2 I_i = -2^q c_k - (1 - 2 x_i) D_i, and a flip changes g_k alone.  Mmax then stays an
        // upper bound of max_k M_k (M_k of the one changed constraint folded in), which keeps the
        // error bound valid; the next item flip recomputes it.
#pragma unroll
        for (int k = 0; k < MC; ++k) {
            if (k >= m) break;
            const int o0 = ip->slack_off[k], o1 = ip->slack_off[k + 1];
            float coef = 1.f;
            for (int i = o0; i < o1; ++i, coef *= 2.f) {
                if ((i & 3) == 0)
                    rw = philox4x32_10(
                        make_uint4((uint32_t)(i >> 2), (uint32_t)t, (uint32_t)chain, iter), key0,
                        key1);
                if ((i & 31) == 0) xw = xs[(i >> 5) * cpb + tid];
                const uint32_t word = word_of(rw, i & 3);
                const float theta = theta_of_word(word);
                const int xi = (xw >> (i & 31)) & 1;
                float acc = sf * 0.f;
                acc = fmaf(-coef, c[k], acc);
                const float Di = __ldg(Dv + i);
                acc = fmaf(xi ? 1.f : -1.f, Di, acc);
                const float z = hb * acc;
                const float y = z + theta;
                const float bound =
                    ez * (coef * Mmax + Di) + kThetaRelErr * fabsf(theta) + kThetaAbsErr;
                int xn;
                if (fabsf(y) > bound) {
                    xn = y > 0.f;
                } else {
                    int32_t ak[MC], g[MC];
#pragma unroll
                    for (int kk = 0; kk < MC; ++kk) {
                        ak[kk] = kk == k ? (int32_t)coef : 0;
                        g[kk] = (int32_t)gf[kk];
                    }
                    xn = decide_exact<MC>(0.f, xi, ak, g, lam, m, sf, sg, psg2, beta,
                                          rho_of_word(word));
                }
                const int d = xn - xi;
                if (d != 0) {
                    xw ^= 1u << (i & 31);
                    gf[k] = fmaf(coef, (float)d, gf[k]);   // exact integers
                    c[k] = fmaf(kappa, gf[k], cA[k]);
                    Mmax = fmaxf(Mmax, fmaf(fabsf(kappa), fabsf(gf[k]), fabsf(cA[k])));
                }
                if ((i & 31) == 31 || i == nprime - 1) xs[(i >> 5) * cpb + tid] = xw;
            }
        }
        if (track) {
            bool feas = true;
#pragma unroll
            for (int k = 0; k < MC; ++k) {
                if (k < m) {
                    const int o0 = ip->slack_off[k], o1 = ip->slack_off[k + 1];
                    long long sv = 0;
                    for (int s = o0; s < o1; ++s)
                        if ((xs[(s >> 5) * cpb + tid] >> (s & 31)) & 1u) sv += 1LL << (s - o0);
                    if ((long long)gf[k] - sv > (long long)ip->fmargin[k]) feas = false;
                }
            }
            if (feas) {
                ++rnf;
                if (ccur < rbest) {
                    rbest = ccur;
                    rsweep = t;
                    if (valid) {
                        uint32_t *rx = a.run_x + ((size_t)j * a.chains + chain) * a.words;
                        for (int w = 0; w < a.words; ++w) rx[w] = w < words ? xs[w * cpb + tid] : 0u;
                    }
                }
            }
        }
        if (a.trace && valid) {
            uint32_t *tr = a.trace + (((size_t)j * a.chains + chain) * a.sweeps + t) * a.words;
            for (int w = 0; w < a.words; ++w) tr[w] = w < words ? xs[w * cpb + tid] : 0u;
        }
    }

    // Readout of the last sample (Sec. III-B): state, cost c(x) = -(sum_i x_i F_i + h^T x)/2
    // (F_i = h_i + (W x)_i), constraint values and items-only feasibility (Sec. IV-A).
    if (!valid) return;
    const size_t cidx = (size_t)j * a.chains + chain;
    long long sumF = 0, sumh = 0;
    for (int w = 0; w < words; ++w) {
        uint32_t bits = xs[w * cpb + tid];
        a.x[cidx * a.words + w] = bits;
        while (bits) {
            const int i = w * 32 + __ffs(bits) - 1;
            bits &= bits - 1u;
            sumh += (long long)__ldg(hF + i);
            sumF += has_w ? (long long)Fs[i * cpb + tid] : (long long)__ldg(hF + i);
        }
    }
    for (int w = words; w < a.words; ++w) a.x[cidx * a.words + w] = 0u;
    a.cost[cidx] = -(sumF + sumh) / 2;
    bool feas = true;
#pragma unroll
    for (int k = 0; k < MC; ++k) {
        if (k < m) {
            const int o0 = ip->slack_off[k], o1 = ip->slack_off[k + 1];
            long long sv = 0;
            for (int s = o0; s < o1; ++s)
                if ((xs[(s >> 5) * cpb + tid] >> (s & 31)) & 1u) sv += 1LL << (s - o0);
            if ((long long)gf[k] - sv > (long long)ip->fmargin[k]) feas = false;
            a.g[cidx * a.m_stride + k] = (long long)gf[k];
        }
    }
    for (int k = m; k < a.m_stride; ++k) a.g[cidx * a.m_stride + k] = 0;
    if (a.feasible) a.feasible[cidx] = feas ? 1 : 0;
    if (track) {
        a.run_cost[cidx] = rbest;
        if (a.run_sweep) a.run_sweep[cidx] = rsweep;
        if (a.run_nfeas) a.run_nfeas[cidx] = rnf;
        if (rsweep < 0)
            for (int w = 0; w < a.words; ++w) a.run_x[cidx * a.words + w] = 0u;
    }
}

}  // namespace
}  // namespace sais
