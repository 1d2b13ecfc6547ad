// sais_blocked_kernel.cuh -- blocked p-bit sampler with the rank-k field update on the tensor cores.
//
// The Gibbs sweep of Sec. III-B stays sequential: spins are visited in index order and each
// decision sees every earlier flip.  What changes is how the objective field
// F_i = h_i + sum_j W_ij x_j follows the flips.  Spins are taken in blocks of K:
//   1. the K decisions of a block are made one after the other on CUDA cores, each flip
//      correcting the F values of the block's later spins (W[blk, blk], k(k-1)/2 products);
//   2. the block's flips Delta (values -1, 0, +1) then update every field at once,
//      F[:, chains] += W[:, blk] Delta[blk, chains], a dense GEMM of N'_pad x K x 128 done by
//      tcgen05.mma in BF16 with FP32 accumulation.  The products and partial sums are
//      integers below 2^24, so the result is exact and equal to the per-flip updates of the
//      plain sampler: both samplers make identical decisions.
//
// Layout (one CTA = 128 chains of one instance; 1 CTA per SM):
//   TMEM   F transposed, lane = chain (MMA row M = 128), column = spin (N = N'_pad), FP32.
//   TMEM   also the MMA's A operand Delta (double buffered, K/2 columns each after F): row =
//          chain, two BF16 values per 32-bit column, written by the chain's thread.
//   SMEM   W as BF16 in the no-swizzle core-matrix layout, column-chunk major:
//          element (j, s) at ((s/8) N'_pad + j) * 16 + (s%8) * 2 bytes, so the K columns of one
//          block form a contiguous K-major operand (LBO = 16 N'_pad, SBO = 128); loaded once
//          per launch by bulk asynchronous copies (TMA engine).  A two-slot ring of noise.
//   Warps  0-3 decide (warp w owns TMEM lanes 32w..32w+31, i.e. its 32 chains); the last of
//          them to finish a block issues the block's MMAs.  Warps 4-7 compute the noise (Philox,
//          atanh) up to two blocks ahead for decision warps 0-3, so that every SM
//          sub-partition has a second warp to issue from while its decision warp waits on a
//          dependency; lane 0 of warp 4 also stages W by bulk copies.  Every mbarrier wait is bounded: on expiry the kernel
//          records SAIS_ETIMEOUT, stops, drains its copies and MMAs, frees TMEM and exits.
#pragma once

#include "sais_device.cuh"
#include "sais_tc.cuh"

namespace sais {
namespace {

constexpr int kLanes = 128;
constexpr int kIssueThread = 128;
constexpr int kThreadsBlocked = 256;   // 4 decision warps, 4 noise warps
constexpr int kNoiseWarp0 = 4;
// Every wait of this kernel is for an event microseconds away (an MMA, a block of decisions,
// a 200 KB copy).  A wait gives up after kWaitCycles SM clock cycles (about 4 s at 2 GHz;
// longer if the clock runs slower), or after `polls` polls when a test asks for a poll bound
// (polls > 0).  The SM cycle counter is a cheap register read, unlike the global timer.
constexpr long long kWaitCycles = 8000000000ll;

__device__ __forceinline__ unsigned long long sm_cycles() {
    return (unsigned long long)clock64();
}

__device__ __forceinline__ bool wait_expired(long long n, long long polls,
                                             unsigned long long t0) {
    return polls > 0 ? n >= polls : (long long)(sm_cycles() - t0) > kWaitCycles;
}

// The clock is read only once a first poll has failed: most waits find their phase complete.
__device__ __forceinline__ bool wait_bounded(uint64_t *bar, uint32_t parity,
                                             volatile int *abort_flag, int32_t *status,
                                             long long polls) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = sm_cycles();
    for (long long n = 0;; ++n) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if (abort_flag && *abort_flag) return false;
        if (wait_expired(n, polls, t0)) {
            if (abort_flag) *abort_flag = 1;
            if (status) atomicExch(status, (int32_t)SAIS_ETIMEOUT);
            return false;
        }
    }
}

// Warp-collective bounded wait: every lane polls and the warp leaves together, either when all
// lanes have observed the phase or when any lane sees the abort flag or the poll limit.
__device__ __forceinline__ bool wait_bounded_warp(uint64_t *bar, uint32_t parity,
                                                  volatile int *abort_flag, int32_t *status,
                                                  long long polls) {
    if (__all_sync(0xffffffffu, tc::mbar_try_wait(bar, parity))) return true;
    const unsigned long long t0 = sm_cycles();
    for (long long n = 0;; ++n) {
        const bool got = tc::mbar_try_wait(bar, parity);
        if (__all_sync(0xffffffffu, got)) return true;
        const bool give_up = *abort_flag != 0 || wait_expired(n, polls, t0);
        if (__any_sync(0xffffffffu, give_up)) {
            if ((threadIdx.x & 31) == 0 && !*abort_flag) {
                *abort_flag = 1;
                if (status) atomicExch(status, (int32_t)SAIS_ETIMEOUT);
            }
            return false;
        }
    }
}

__device__ __forceinline__ uint32_t bf16_pm1(int d) {
    return d > 0 ? 0x3F80u : (d < 0 ? 0xBF80u : 0u);
}

template <int K>
__device__ __forceinline__ void load_block_fields(uint32_t taddr, float (&Fr)[K]) {
    if constexpr (K == 32) {
        tc::tmem_ld32(taddr, Fr);
    } else {
        tc::tmem_ld16(taddr, Fr);
    }
}

// kStream: W is not resident; the K columns of each block (one contiguous range of the
// column-chunk-major image) are copied into a ring of kRing tile slots, two blocks ahead.
// kHiLo: W = W_hi + W_lo, both BF16 and exact for |W| < 2^16; two MMAs per block into the same
// accumulator, and the in-block correction adds both terms.
template <int MC, int K, bool kStream, bool kHiLo>
__global__ void __launch_bounds__(kThreadsBlocked, 1)
    blocked_sampler_kernel(SampleArgs a, int32_t *status, long long dec_wait_polls,
                           uint32_t tmem_cols) {
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int kPreM = MC < 2 ? MC : 2;   // constraint columns in the per-spin record
    constexpr uint32_t kRing = 3;
    const int j = a.work ? a.work[2 * blockIdx.x] : (int)blockIdx.y;
    const int grp = a.work ? a.work[2 * blockIdx.x + 1] : (int)blockIdx.x;
    if (!SAIS_DCHECK(status, j >= 0 && j < a.count && grp >= 0 && grp * kLanes < a.chains))
        return;
    const InstDev *__restrict__ ip = a.inst + j;
    const int m = ip->m, nprime = ip->nprime, npad = ip->npad, words = ip->words;
    const int nb = (nprime + K - 1) / K;
    const uint32_t wbytes = (uint32_t)npad * (uint32_t)npad * 2u;
    const uint32_t tile_bytes = (uint32_t)(K / 8) * (uint32_t)npad * 16u;   // one term, one block
    const uint32_t slot_bytes = tile_bytes * (kHiLo ? 2u : 1u);
    const uint32_t wregion = kStream ? kRing * slot_bytes : wbytes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    unsigned char *Wsm = smem;   // resident image, or the tile ring
    uint32_t *xs = reinterpret_cast<uint32_t *>(smem + wregion);
    float *thbuf = reinterpret_cast<float *>(xs + words * kLanes);   // [2][K][128] noise ring
    uint64_t *bars = reinterpret_cast<uint64_t *>(thbuf + 2 * K * kLanes);
    // bars: 0 = W staged, 1 = never completed (fault-injection test of the timeout path),
    // 2 = unused, 3..6 = drain of decision warp 0..3,
    // 7..14 = noise slot written (2 q + slot), 15..22 = noise slot consumed (2 q + slot),
    // 23..25 = W tile slot filled, 26..28 = W tile slot free again (its block's MMAs done),
    // 29 = the block's MMAs done
    uint32_t *arrivals = reinterpret_cast<uint32_t *>(bars + 30);   // [2] decision warps done
    uint32_t *tmem_slot = arrivals + 2;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    // Debug builds: F and the Delta slots within the CTA's TMEM, the layout within its shared
    // memory (every thread evaluates the same values).
    if (!SAIS_DCHECK(status, (uint32_t)(npad + K) <= tmem_cols &&
                                 (uint32_t)(reinterpret_cast<unsigned char *>(
                                                const_cast<int *>(abort_flag) + 1) -
                                            smem) <= dynamic_smem_bytes()))
        return;
    if (threadIdx.x == kIssueThread) {
        for (int i = 0; i < 30; ++i) tc::mbar_init(&bars[i], 1);
        arrivals[0] = arrivals[1] = 0u;
        *abort_flag = 0;
        tc::fence_mbar_init();
        tc::fence_proxy_async_smem();
    }
    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, tmem_cols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t iter = a.iter_dev ? *a.iter_dev : a.iter;

    if (warp >= kNoiseWarp0) {
        // Noise warps: warp 4+q produces theta = atanh(rho) for the chains of decision warp q,
        // up to two blocks ahead, into a two-slot ring.  Lane 0 of warp 4 stages W.
        const int q = warp - kNoiseWarp0;
        const int r = q * 32 + lane;
        const uint32_t chain = (uint32_t)(grp * kLanes + r);
        const uint64_t seed = a.seed + (uint64_t)j;
        const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
        const uint32_t total = (uint32_t)a.sweeps * (uint32_t)nb;
        if (!kStream && q == 0 && lane == 0) {
            tc::mbar_expect_tx(&bars[0], wbytes);
            const unsigned char *src = reinterpret_cast<const unsigned char *>(ip->Wbf);
            for (uint32_t off = 0; off < wbytes; off += 32768u)
                tc::bulk_g2s(Wsm + off, src + off, min(32768u, wbytes - off), &bars[0]);
        }
        uint32_t tiles_issued = 0;
        for (uint32_t it = 0; it < total; ++it) {
            const uint32_t slot = it & 1u;
            if (it >= 2 && !wait_bounded_warp(&bars[15 + 2 * q + slot], ((it >> 1) + 1u) & 1u,
                                              abort_flag, status, 0))
                break;
            if (kStream && q == 0) {
                // W tile of block `it` into slot it % kRing, once that slot's previous block
                // (it - kRing) has had its MMAs completed.
                bool okt = true;
                if (lane == 0) {
                    const uint32_t ts = it % kRing;
                    if (it >= kRing)
                        okt = wait_bounded(&bars[26 + ts], ((it / kRing) - 1u) & 1u, abort_flag,
                                           status, 0);
                    if (okt) {
                        const uint32_t b = it % (uint32_t)nb;
                        unsigned char *dst = Wsm + ts * slot_bytes;
                        tc::mbar_expect_tx(&bars[23 + ts], slot_bytes);
                        tc::bulk_g2s(dst, reinterpret_cast<const unsigned char *>(ip->Wbf) +
                                              (size_t)b * tile_bytes,
                                     tile_bytes, &bars[23 + ts]);
                        if (kHiLo)
                            tc::bulk_g2s(dst + tile_bytes,
                                         reinterpret_cast<const unsigned char *>(ip->Wbf_lo) +
                                             (size_t)b * tile_bytes,
                                         tile_bytes, &bars[23 + ts]);
                        ++tiles_issued;
                    }
                }
                if (__shfl_sync(0xffffffffu, okt ? 1 : 0, 0) == 0) break;
            }
            const uint32_t t = it / (uint32_t)nb;
            const int s0 = (int)(it % (uint32_t)nb) * K;
            float *tb = thbuf + slot * K * kLanes;
#pragma unroll
            for (int g4 = 0; g4 < K / 4; ++g4) {
                const uint4 rw = philox4x32_10(
                    make_uint4((uint32_t)((s0 >> 2) + g4), t, chain, iter), key0, key1);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    // Spins past N' (block padding) get a threshold that keeps them at 0.
                    const bool real = s0 + 4 * g4 + e < nprime;
                    tb[(4 * g4 + e) * kLanes + r] = real ? theta_of_word(word_of(rw, e)) : -1e30f;
                }
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&bars[7 + 2 * q + slot]);
        }
        // The staging copies complete before shared memory is released.
        if (q == 0 && lane == 0) {
            if (!kStream) {
                wait_bounded(&bars[0], 0, nullptr, status, 0);
            } else {
                for (uint32_t ts = 0; ts < kRing && ts < tiles_issued; ++ts) {
                    const uint32_t uses = (tiles_issued - ts + kRing - 1u) / kRing;
                    wait_bounded(&bars[23 + ts], (uses - 1u) & 1u, nullptr, status, 0);
                }
            }
        }
        __syncwarp();
    } else {
        const int r = threadIdx.x;
        const int chain = grp * kLanes + r;
        const bool valid = chain < (a.inst_chains ? a.inst_chains[j] : a.chains);
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        const uint64_t seed = a.seed + (uint64_t)j;
        const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
        const float sf = ip->sigma_f, sg = ip->sigma_g, kappa = ip->kappa;
        const double psg2 = ip->psg2;
        const float *__restrict__ hF = ip->hF;
        const int32_t *__restrict__ acol = ip->acol;
        const float *__restrict__ Dv = ip->D;
        const float *__restrict__ asum = ip->asum;
        const float *lam = a.lambda + (size_t)j * a.m_stride;

        // x = 0 and F = h (Sec. III-B: every run starts from x = 0).
        for (int w = 0; w < words; ++w) xs[w * kLanes + r] = 0u;
        for (int c0 = 0; c0 < npad; c0 += 32) {
            float v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = __ldg(hF + c0 + i);
            tc::tmem_st32(lane_addr + (uint32_t)c0, v);
        }
        tc::tc_fence_before();

        int32_t g[MC];
        float c[MC], cA[MC];
        float Mmax = 0.f;
#pragma unroll
        for (int k = 0; k < MC; ++k) {
            if (k < m) {
                cA[k] = __double2float_rn((double)sg * (double)lam[k]);
                g[k] = -ip->b[k];
                c[k] = fmaf(kappa, (float)g[k], cA[k]);
                Mmax = fmaxf(Mmax, fmaf(fabsf(kappa), fabsf((float)g[k]), fabsf(cA[k])));
            } else {
                cA[k] = 0.f;
                g[k] = 0;
                c[k] = 0.f;
            }
        }
        // The constraint values as FP32 too (exact: |g| < 2^24, checked at creation), so that the
        // decision chain updates them and c_k without integer <-> float conversions; the int32
        // copy is refreshed from them where it is needed (exact re-runs, readout).
        float gf[MC];
#pragma unroll
        for (int k = 0; k < MC; ++k) gf[k] = (float)g[k];
        const float errk = field_err_factor(m);
        // Fault-injection test (dec_wait_polls > 0): wait on a barrier nothing completes, so the
        // bound expires and the kernel takes its timeout path.
        bool ok = dec_wait_polls > 0
                      ? wait_bounded_warp(&bars[1], 0, abort_flag, status, dec_wait_polls)
                      : true;
        if (ok && !kStream) ok = wait_bounded_warp(&bars[0], 0, abort_flag, status, 0);
        // Best feasible sweep-end state of the run (a.run_cost set): at a sweep end where a
        // chain of the warp is feasible, the warp waits for the sweep's last MMA and reads the
        // cost c(x) = -(sum_i x_i F_i + h^T x)/2 off the fields in TMEM; the block path is
        // untouched.
        const bool track = a.run_cost != nullptr;
        long long rbest = LLONG_MAX;
        int rsweep = -1, rnf = 0;
        uint32_t it = 0;
        float th[K];
        for (int t = 0; ok && t < a.sweeps; ++t) {
            const float beta = beta_of_sweep(a.beta_max, t, a.sweeps);
            const float hb = 0.5f * beta;
            const float ez = hb * errk;
            for (int b = 0; b < nb; ++b) {
                const int s0 = b * K;
                // Noise of the block, written by this warp's partner noise warp.
                const uint32_t slot = it & 1u;
                if (!wait_bounded_warp(&bars[7 + 2 * warp + slot], (it >> 1) & 1u, abort_flag,
                                       status, dec_wait_polls)) {
                    ok = false;
                    break;
                }
#pragma unroll
                for (int ii = 0; ii < K; ++ii) th[ii] = thbuf[(slot * K + ii) * kLanes + r];
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&bars[15 + 2 * warp + slot]);
                // W columns of the block: the resident image, or the tile slot of this block.
                const unsigned char *wblk =
                    kStream ? Wsm + (it % kRing) * slot_bytes
                            : Wsm + (size_t)(s0 >> 3) * (size_t)npad * 16u;
                if (kStream && !wait_bounded_warp(&bars[23 + it % kRing], (it / kRing) & 1u,
                                                  abort_flag, status, dec_wait_polls)) {
                    ok = false;
                    break;
                }
                // Per-spin constants of the block, loaded together before the sequential loop
                // and before the wait for the previous block's MMAs, which they overlap
                // (spins past N' read the zero padding of the arrays).
                float Dp[K], Sp[K];
                float Ap[K][kPreM];
#pragma unroll
                for (int ii = 0; ii < K; ++ii) {
                    const float4 sc = __ldg(ip->spinc + s0 + ii);
                    Ap[ii][0] = sc.x;
                    Dp[ii] = sc.y;
                    Sp[ii] = sc.z;
                    if (kPreM > 1) Ap[ii][kPreM > 1 ? 1 : 0] = sc.w;
                }
                if (it > 0) {
                    // This block's fields: the previous block's MMAs are done (MMAs complete in
                    // issue order, so those of every earlier block too, which also frees this
                    // block's Delta slot, last used two blocks ago).
                    if (!wait_bounded_warp(&bars[29], (it - 1u) & 1u, abort_flag, status,
                                           dec_wait_polls)) {
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                }
                float Fr[K];
                load_block_fields<K>(lane_addr + (uint32_t)s0, Fr);
                const int wi = s0 >> 5, sb = s0 & 31;
                uint32_t xw = xs[wi * kLanes + r];
                const uint32_t xold = xw;
                // Block-start chain state, kept for an exact re-run of the block.
                float gf0[MC], cb[MC];
                const float M0 = Mmax;
#pragma unroll
                for (int k = 0; k < MC; ++k) {
                    gf0[k] = gf[k];
                    cb[k] = c[k];
                }
                bool near_tie = false;
#pragma unroll
                for (int ii = 0; ii < K; ++ii) {
                    const int s = s0 + ii;
                    // Row s of the block's W columns (only the part right of spin ii is used):
                    // loaded ahead of the decision so that it is ready if any chain flips.
                    // W streamed (K = 16): the block's 16 x 16 diagonal tile of W in FP32
                    // (exact, hi and lo already added; the same address for every lane), the
                    // quads right of spin ii -- measured faster than the BF16 tile columns here.
                    // W resident: its BF16 columns in shared memory (faster there).
                    uint4 wrow[K / 8], wrlo[K / 8];
                    float4 wq[4];
                    if constexpr (K == 16 && kStream) {
                        const float4 *wd4 = reinterpret_cast<const float4 *>(
                            ip->Wdiag + (size_t)(s0 / 16) * 256 + ii * 16);
#pragma unroll
                        for (int q = (ii + 1) >> 2; q < 4; ++q) wq[q] = __ldg(wd4 + q);
                    } else {
#pragma unroll
                        for (int cc = (ii + 1) >> 3; cc < K / 8; ++cc) {
                            wrow[cc] = *reinterpret_cast<const uint4 *>(
                                wblk + ((size_t)cc * npad + s) * 16);
                            if (kHiLo)
                                wrlo[cc] = *reinterpret_cast<const uint4 *>(
                                    wblk + tile_bytes + ((size_t)cc * npad + s) * 16);
                        }
                    }
                    {
                        const float Fi = Fr[ii];
                        const int xi = (xw >> (sb + ii)) & 1;
                        float akf[MC];
                        float acc = sf * Fi;
                        const float tabs = fabsf(acc);
#pragma unroll
                        for (int k = 0; k < MC; ++k) {
                            if (k < kPreM)
                                akf[k] = Ap[ii][k < kPreM ? k : 0];
                            else
                                akf[k] = (k < m) ? (float)__ldg(acol + (size_t)s * m + k) : 0.f;
                            acc = fmaf(-akf[k], c[k], acc);
                        }
                        const float Di = Dp[ii];
                        acc = fmaf(xi ? 1.f : -1.f, Di, acc);
                        const float z = hb * acc;
                        const float theta = th[ii];
                        const float y = z + theta;
                        const float bound = ez * (tabs + Sp[ii] * Mmax + Di) +
                                            kThetaRelErr * fabsf(theta) + kThetaAbsErr;
                        // A decision the FP32 bound cannot settle is only flagged here; the
                        // warp then re-runs the block below with the FP64 path.
                        near_tie |= !(fabsf(y) > bound);
                        // The flip d = x_new - x_i in {-1, 0, +1}, kept as FP32.
                        const float df = (y > 0.f ? 1.f : 0.f) - (xi ? 1.f : 0.f);
                        // Constraint state follows the flip without a branch (d = 0 leaves every
                        // value bit-identical).
                        xw ^= (uint32_t)(df != 0.f) << (sb + ii);
                        Mmax = 0.f;
#pragma unroll
                        for (int k = 0; k < MC; ++k) {
                            if (k < m) {
                                gf[k] = fmaf(akf[k], df, gf[k]);   // exact integers
                                c[k] = fmaf(kappa, gf[k], cA[k]);
                                Mmax = fmaxf(Mmax, fmaf(fabsf(kappa), fabsf(gf[k]), fabsf(cA[k])));
                            }
                        }
                        if (ii + 1 < K) {
                            // In-block correction F_jj += W[s, s0+jj] d for the block's later
                            // spins (row s of the block's W columns is contiguous per 8 columns).
                            // The next spin's field is on the dependency chain: corrected
                            // unconditionally (d = 0 adds an exact zero); the others only when a
                            // chain of the warp flipped.
                            // BF16 value of column jj of the row (jj is a compile-time
                            // constant after unrolling; no local arrays, so nothing goes to the
                            // stack)
                            auto half = [](const uint4 &v, int e) -> float {
                                const int q = e >> 1;
                                const uint32_t u = q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
                                return __uint_as_float((e & 1) ? (u & 0xFFFF0000u) : (u << 16));
                            };
                            auto wcol = [&](int jj) -> float {
                                if constexpr (K == 16 && kStream) {
                                    const float4 &v = wq[jj >> 2];
                                    const int e = jj & 3;
                                    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
                                } else {
                                    float w = half(wrow[jj >> 3], jj & 7);
                                    if (kHiLo) w += half(wrlo[jj >> 3], jj & 7);   // exact
                                    return w;
                                }
                            };
                            Fr[ii + 1] = fmaf(df, wcol(ii + 1), Fr[ii + 1]);
                            if (ii + 2 < K && __any_sync(0xffffffffu, df != 0.f)) {
#pragma unroll
                                for (int jj = ii + 2; jj < K; ++jj)
                                    Fr[jj] = fmaf(df, wcol(jj), Fr[jj]);
                            }
                        }
                    }
                }
                if (__any_sync(0xffffffffu, near_tie)) {
                    // Exact re-run of the block for the whole warp, from its start state: F from
                    // TMEM (this block's MMA is not issued yet) plus the block's earlier flips, the
                    // noise recomputed, the same FP32 evaluation, and FP64 where the bound cannot
                    // settle the decision.  Decisions outside near-ties come out as before.
                    xw = xold;
                    Mmax = M0;
#pragma unroll
                    for (int k = 0; k < MC; ++k) {
                        g[k] = (int32_t)gf0[k];
                        c[k] = cb[k];
                    }
#pragma unroll 1
                    for (int ii = 0; ii < K; ++ii) {
                        const int s = s0 + ii;
                        uint32_t fv;
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                                     : "=r"(fv)
                                     : "r"(lane_addr + (uint32_t)s));
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        float Fi = __uint_as_float(fv);
                        uint32_t fl = ((xw ^ xold) >> sb) & ((1u << ii) - 1u);
                        while (fl) {
                            const int i2 = __ffs(fl) - 1;
                            fl &= fl - 1u;
                            const int d2 = (int)((xw >> (sb + i2)) & 1u) -
                                           (int)((xold >> (sb + i2)) & 1u);
                            const size_t off = ((size_t)(i2 >> 3) * npad + s) * 16 + (i2 & 7) * 2;
                            const uint16_t wb = *reinterpret_cast<const uint16_t *>(wblk + off);
                            float w = __uint_as_float((uint32_t)wb << 16);
                            if (kHiLo)
                                w += __uint_as_float(
                                    (uint32_t)*reinterpret_cast<const uint16_t *>(
                                        wblk + tile_bytes + off)
                                    << 16);
                            Fi = fmaf((float)d2, w, Fi);
                        }
                        const int xi = (xw >> (sb + ii)) & 1;
                        int32_t ak[MC];
                        float acc = sf * Fi;
                        const float tabs = fabsf(acc);
#pragma unroll
                        for (int k = 0; k < MC; ++k) {
                            ak[k] = (k < m) ? __ldg(acol + (size_t)s * m + k) : 0;
                            acc = fmaf(-(float)ak[k], c[k], acc);
                        }
                        const float Di = __ldg(Dv + s);
                        acc = fmaf(xi ? 1.f : -1.f, Di, acc);
                        const float z = hb * acc;
                        const uint4 rw = philox4x32_10(
                            make_uint4((uint32_t)(s >> 2), (uint32_t)t, (uint32_t)chain, iter),
                            key0, key1);
                        const float theta =
                            s < nprime ? theta_of_word(word_of(rw, s & 3)) : -1e30f;
                        const float y = z + theta;
                        const float bound = ez * (tabs + __ldg(asum + s) * Mmax + Di) +
                                            kThetaRelErr * fabsf(theta) + kThetaAbsErr;
                        int xn = y > 0.f;
                        if (!(fabsf(y) > bound)) {
                            const float rho = rho_of_word(word_of(rw, s & 3));
                            xn = decide_exact<MC>(Fi, xi, ak, g, lam, m, sf, sg, psg2, beta, rho);
                        }
                        const int d = xn - xi;
                        xw ^= (uint32_t)(d != 0) << (sb + ii);
                        Mmax = 0.f;
#pragma unroll
                        for (int k = 0; k < MC; ++k) {
                            if (k < m) {
                                g[k] += ak[k] * d;
                                c[k] = fmaf(kappa, (float)g[k], cA[k]);
                                Mmax = fmaxf(Mmax, fmaf(fabsf(kappa), fabsf((float)g[k]),
                                                        fabsf(cA[k])));
                            }
                        }
                    }
#pragma unroll
                    for (int k = 0; k < MC; ++k) gf[k] = (float)g[k];
                }
                xs[wi * kLanes + r] = xw;
                // Delta of the block (BF16 -1, 0, +1) into this chain's TMEM row of the MMA's A
                // operand (columns N'_pad + slot K/2 ..); the last decision warp to finish the
                // block issues its MMAs: F[:, chains] += W[:, blk] Delta[blk, chains].
                {
                    const uint32_t a_col = (uint32_t)npad + (it & 1u) * (uint32_t)(K / 2);
                    uint32_t pk[K / 2];
#pragma unroll
                    for (int e2 = 0; e2 < K / 2; ++e2) {
                        const int i0 = sb + 2 * e2;
                        const int d0 = (int)((xw >> i0) & 1u) - (int)((xold >> i0) & 1u);
                        const int d1 = (int)((xw >> (i0 + 1)) & 1u) - (int)((xold >> (i0 + 1)) & 1u);
                        pk[e2] = bf16_pm1(d0) | (bf16_pm1(d1) << 16);
                    }
#pragma unroll
                    for (int h8 = 0; h8 < K / 16; ++h8) {
                        uint32_t v8[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) v8[e] = pk[8 * h8 + e];
                        tc::tmem_st8(lane_addr + a_col + 8u * (uint32_t)h8, v8);
                    }
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        __threadfence_block();
                        const bool last = (atomicAdd(&arrivals[it & 1u], 1u) & 3u) == 3u;
                        if (last) {
                            __threadfence_block();
                            tc::tc_fence_after();
                            const uint32_t lbo_b = (uint32_t)npad * 16u;
                            const uint32_t w_base = tc::smem_u32(wblk);
                            // Columns [c0, c1) of F += W[., blk] Delta, in MMAs of <= 256 columns.
                            auto mma_cols = [&](int c0, int c1) {
#pragma unroll
                                for (int term = 0; term < (kHiLo ? 2 : 1); ++term) {
#pragma unroll
                                    for (int ks = 0; ks < K / 16; ++ks) {
                                        for (int j0 = c0; j0 < c1; j0 += 256) {
                                            const int nr = min(256, c1 - j0);
                                            const uint64_t bd = tc::smem_desc(
                                                w_base + (uint32_t)term * tile_bytes +
                                                    (uint32_t)ks * 2u * lbo_b + (uint32_t)j0 * 16u,
                                                lbo_b, 128u);
                                            tc::mma_bf16_tmem_a(
                                                tmem + (uint32_t)j0, tmem + a_col + 8u * (uint32_t)ks,
                                                bd, tc::idesc_bf16_f32(128, (uint32_t)nr), 1u);
                                        }
                                    }
                                }
                            };
                            // All columns in one go.  (Issuing the next block's columns first, so
                            // that its decisions wait for a narrow MMA only, measured slower: the
                            // extra MMAs and commits cost more than the wait they save.)
                            mma_cols(0, npad);
                            tc::mma_commit(&bars[29]);
                            if (kStream) tc::mma_commit(&bars[26 + it % kRing]);
                        }
                    }
                    __syncwarp();
                }
                ++it;
            }
            if (ok && track) {
                bool feas = true;
#pragma unroll
                for (int k = 0; k < MC; ++k) {
                    if (k < m) {
                        const int o0 = ip->slack_off[k], o1 = ip->slack_off[k + 1];
                        long long sv = 0;
                        for (int s = o0; s < o1; ++s)
                            if ((xs[(s >> 5) * kLanes + r] >> (s & 31)) & 1u) sv += 1LL << (s - o0);
                        if ((long long)gf[k] - sv > (long long)ip->fmargin[k]) feas = false;
                    }
                }
                long long cost = LLONG_MAX;
                if (__any_sync(0xffffffffu, feas)) {
                    // F is current once the sweep's last MMA is done (the next block waits for
                    // the same phase; no later one can complete before this warp's next block).
                    if (!wait_bounded_warp(&bars[29], (it - 1u) & 1u, abort_flag, status,
                                           dec_wait_polls)) {
                        ok = false;
                    } else {
                        tc::tc_fence_after();
                        long long sumF = 0, sumh = 0;
                        for (int c0 = 0; c0 < npad; c0 += 32) {
                            float v[32];
                            tc::tmem_ld32(lane_addr + (uint32_t)c0, v);
                            const uint32_t bits = c0 < words * 32 ? xs[(c0 >> 5) * kLanes + r] : 0u;
                            int32_t pf = 0, ph = 0;   // |F|, |h| < 2^24: 32 terms fit int32
#pragma unroll
                            for (int i = 0; i < 32; ++i) {
                                if ((bits >> i) & 1u) {
                                    pf += __float2int_rz(v[i]);
                                    ph += __float2int_rz(__ldg(hF + c0 + i));
                                }
                            }
                            sumF += pf;
                            sumh += ph;
                        }
                        cost = -(sumF + sumh) / 2;
                    }
                }
                if (ok && feas) {
                    ++rnf;
                    if (cost < rbest) {
                        rbest = cost;
                        rsweep = t;
                        if (valid) {
                            uint32_t *rx = a.run_x + ((size_t)j * a.chains + chain) * a.words;
                            for (int w = 0; w < a.words; ++w)
                                rx[w] = w < words ? xs[w * kLanes + r] : 0u;
                        }
                    }
                }
            }
            if (ok && a.trace && valid) {
                uint32_t *tr = a.trace + (((size_t)j * a.chains + chain) * a.sweeps + t) * a.words;
                for (int w = 0; w < a.words; ++w) tr[w] = w < words ? xs[w * kLanes + r] : 0u;
            }
        }
        // Drain: every MMA of the CTA completes before the readout and the TMEM release.  Each
        // decision warp's lane 0 commits the MMAs it issued (any of them may have issued some);
        // every warp waits for all four, bounded but not cut short by an abort.
        if (lane == 0) tc::mma_commit(&bars[3 + warp]);
        __syncwarp();
        bool drained = true;
        if (lane == 0)
            for (int w = 0; w < 4; ++w)
                drained = wait_bounded(&bars[3 + w], 0, nullptr, status, 0) && drained;
        drained = __shfl_sync(0xffffffffu, drained ? 1 : 0, 0) != 0;
        tc::tc_fence_after();
        if (ok && drained) {
            // Readout of the last sample: cost -(sum_i x_i F_i + h^T x)/2, g, feasibility.  The
            // TMEM loads are warp-collective, so every lane takes part; only valid chains store.
            long long sumF = 0, sumh = 0;
            for (int c0 = 0; c0 < npad; c0 += 32) {
                float v[32];
                tc::tmem_ld32(lane_addr + (uint32_t)c0, v);
                const uint32_t bits = c0 < words * 32 ? xs[(c0 >> 5) * kLanes + r] : 0u;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    if ((bits >> i) & 1u) {
                        sumF += (long long)v[i];
                        sumh += (long long)__ldg(hF + c0 + i);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < MC; ++k) g[k] = (int32_t)gf[k];
            if (valid) {
                const size_t cidx = (size_t)j * a.chains + chain;
                for (int w = 0; w < a.words; ++w)
                    a.x[cidx * a.words + w] = w < words ? xs[w * kLanes + r] : 0u;
                a.cost[cidx] = -(sumF + sumh) / 2;
                bool feas = true;
#pragma unroll
                for (int k = 0; k < MC; ++k) {
                    if (k < m) {
                        const int o0 = ip->slack_off[k], o1 = ip->slack_off[k + 1];
                        long long sv = 0;
                        for (int s = o0; s < o1; ++s)
                            if ((xs[(s >> 5) * kLanes + r] >> (s & 31)) & 1u) sv += 1LL << (s - o0);
                        if ((long long)g[k] - sv > (long long)ip->fmargin[k]) feas = false;
                        a.g[cidx * a.m_stride + k] = g[k];
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
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, tmem_cols);
    }
}

template <int MC, int K, bool S, bool H>
cudaError_t launch_k(const SampleArgs &a, int32_t *status, long long polls, size_t smem,
                     uint32_t cols, cudaStream_t s) {
    auto kern = blocked_sampler_kernel<MC, K, S, H>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid = a.work ? dim3(a.nwork, 1) : dim3((a.chains + kLanes - 1) / kLanes, a.count);
    kern<<<grid, kThreadsBlocked, smem, s>>>(a, status, polls, cols);
    return cudaGetLastError();
}

template <int K, bool S, bool H>
cudaError_t launch_mc(const SampleArgs &a, int max_m, int32_t *status, long long polls,
                      size_t smem, uint32_t cols, cudaStream_t s) {
    if (max_m <= 1) return launch_k<1, K, S, H>(a, status, polls, smem, cols, s);
    if (max_m <= 2) return launch_k<2, K, S, H>(a, status, polls, smem, cols, s);
    if (max_m <= 4) return launch_k<4, K, S, H>(a, status, polls, smem, cols, s);
    return launch_k<8, K, S, H>(a, status, polls, smem, cols, s);   // the host admits m <= 8
}

}  // namespace
}  // namespace sais
