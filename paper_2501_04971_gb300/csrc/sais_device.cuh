// sais_device.cuh -- device building blocks of the p-bit sampler (Sec. III-B, Eq. 9-10).
//
// The decision of Eq. 10, m_i = sign(tanh(beta I_i) + rho), is taken as
//     x_i = 1  iff  beta I_i + atanh(rho) > 0,
// which is the same test (tanh is increasing; atanh(-rho) = -atanh(rho)) with the
// transcendental moved onto the noise, which does not depend on the chain state.  beta I_i is
// evaluated in FP32 together with a rigorous bound on its error; when |beta I + atanh(rho)| does
// not exceed the bound, the decision is re-evaluated in FP64 as tanh(beta I) + rho > 0.  The
// result is the decision exact arithmetic on the FP32 scalars gives, except for ties within
// FP64 rounding.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include <climits>

#include "sais_internal.h"

namespace sais {

// Debug builds (compiled with SAIS_DEBUG=1): device-side checks of indices and sizes that the
// host's validation makes true by construction.  A failed check records SAIS_EBOUNDS and its
// source line in the problem's status words (status[0], status[1]; the first failure wins) and
// the caller skips the access; release builds compile the checks to `true`.
#if defined(SAIS_DEBUG) && SAIS_DEBUG
static __device__ __noinline__ void dcheck_fail(int32_t *status, int line) {
    if (status && atomicCAS(status, 0, (int32_t)SAIS_EBOUNDS) == 0)
        atomicExch(status + 1, (int32_t)line);
}
#define SAIS_DCHECK(status, cond) ((cond) ? true : (::sais::dcheck_fail((status), __LINE__), false))
#else
#define SAIS_DCHECK(status, cond) true
#endif

// Bytes of dynamic shared memory this launch has.
__device__ __forceinline__ uint32_t dynamic_smem_bytes() {
    uint32_t v;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32 -> 64-bit
// products of counter words 0 and 2 with the round multipliers; the high halves are xor-ed
// with the other counter word and the round key, which advances by the Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// rand(-1,1) of Eq. 10: rho = (2v+1)/2^24 - 1 with v = word >> 8, an odd multiple of 2^-24;
// the integer 2v+1-2^24 has magnitude < 2^24, so the FP32 value is exact.
__device__ __forceinline__ float rho_of_word(uint32_t w) {
    const int32_t k = (int32_t)(2u * (w >> 8) + 1u) - (1 << 24);
    return (float)k * 0x1p-24f;
}

__device__ __forceinline__ uint32_t word_of(const uint4 &r, int q) {
    return q == 0 ? r.x : (q == 1 ? r.y : (q == 2 ? r.z : r.w));
}

// beta_t = beta_max t / (T-1) in FP64, rounded once to FP32 (linear schedule of Sec. III-B).
__device__ __forceinline__ float beta_of_sweep(float beta_max, int t, int T) {
    if (T <= 1) return beta_max;
    return __double2float_rn(__ddiv_rn(__dmul_rn((double)beta_max, (double)t), (double)(T - 1)));
}

// theta = atanh(rho) for rho = (2v+1)/2^24 - 1 (v = word >> 8).  With u = (1+rho)/2 =
// (2v+1)/2^25 and 1-u = (2^25-2v-1)/2^25 (both formed from exact integers and scaled by a power
// of two), atanh(rho) = (1/2) ln(u/(1-u)) = (ln 2 / 2)(log2 u - log2(1-u)).  log2 is the
// hardware approximation (lg2.approx.f32).  Both logarithms are of numbers in (0, 1) whose
// ratio is the quantity of interest, so there is no cancellation near rho = 0.
__device__ __forceinline__ float theta_of_word(uint32_t w) {
    const uint32_t v = w >> 8;
    const float u = (float)(2u * v + 1u) * 0x1p-25f;
    const float um = (float)((1u << 25) - 2u * v - 1u) * 0x1p-25f;
    float lu, lum;
    asm("lg2.approx.f32 %0, %1;" : "=f"(lu) : "f"(u));
    asm("lg2.approx.f32 %0, %1;" : "=f"(lum) : "f"(um));
    return 0.34657359028f * (lu - lum);
}

// Bound on |theta_of_word(w) - atanh(rho)|: kThetaAbsErr + kThetaRelErr |theta|.  The noise takes
// 2^24 distinct values; a GPU test evaluates all of them against FP64 atanh and checks the
// bound (measured maximum reported there).
constexpr float kThetaAbsErr = 0x1p-20f;
constexpr float kThetaRelErr = 0x1p-21f;

// Error factor of the FP32 field: the evaluation below has at most m + 7 roundings weighted by
// the magnitudes it adds up (derivation in sais_plain.cu); (m + 12) u with u = 2^-24 and a
// further 1/16 margin for the rounding of the bound itself.
__host__ __device__ inline float field_err_factor(int m) {
    return (float)(m + 12) * 0x1p-24f * 1.0625f;
}

// FP64 re-evaluation of Eq. 10 for one spin (rarely taken).  The caller passes the integer
// part G = sum_k a_ki (2 g_k + a_ki (1 - 2 x_i)) (exact, int64) and the multiplier part
// lin = sum_k a_ki sigma_g lambda_k; then
//   2 I_i = sigma_f F_i - lin - P sigma_g^2 G,   x_i = [tanh(beta I_i) + rho > 0].
static __device__ __noinline__ bool decide_fp64(float Fi, double lin, long long G, float sigma_f,
                                         double psg2, float beta, float rho) {
    double acc = __dmul_rn((double)sigma_f, (double)Fi);
    acc = __dsub_rn(acc, lin);
    acc = __dsub_rn(acc, __dmul_rn(psg2, (double)G));
    const double z = __dmul_rn(0.5 * (double)beta, acc);
    return tanh(z) + (double)rho > 0.0;
}

// The exact-path inputs G and lin for spin i of one chain (see decide_fp64).
template <int MC>
__device__ __forceinline__ bool decide_exact(float Fi, int xi, const int32_t (&a)[MC],
                                             const int32_t (&g)[MC], const float *lam, int m,
                                             float sigma_f, float sigma_g, double psg2,
                                             float beta, float rho) {
    long long G = 0;
    double lin = 0.0;
#pragma unroll
    for (int k = 0; k < MC; ++k) {
        if (k < m) {
            G += (long long)a[k] * (2LL * g[k] + (long long)a[k] * (1 - 2 * xi));
            lin = __dadd_rn(lin, __dmul_rn((double)a[k],
                                           __dmul_rn((double)sigma_g, (double)__ldg(lam + k))));
        }
    }
    return decide_fp64(Fi, lin, G, sigma_f, psg2, beta, rho);
}

}  // namespace sais
