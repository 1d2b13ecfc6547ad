// sais_pair.cu -- the blocked p-bit sampler on a pair of CTAs (a thread-block cluster of two), for
// instances whose objective field does not fit one SM's tensor memory.
//
// The blocked sampler keeps F (objective field, FP32 exact integers) for 128 chains in TMEM with
// one column per spin, so one CTA holds at most 512 spins.  Here the item columns are split in
// two halves, [0, h) in CTA 0 and [h, n_pad) in CTA 1 of the cluster; both CTAs run the same 128
// chains.  The Gibbs sweep of Sec. III-B stays sequential, spin by spin:
//   * a block of K = 16 spins inside CTA p's half is decided by CTA p (it holds their fields);
//     its flips Delta (BF16 -1/0/+1, the MMA's A operand, 128 x 16) are written into both
//     CTAs' shared memory (the peer's through distributed shared memory) and the peer is
//     signalled with remote mbarrier arrivals;
//   * both CTAs then apply the rank-16 update to their own half of F with tcgen05.mma,
//     F[:, half] += W[half, blk] Delta[blk, :], W streamed per block through a tile ring; each
//     CTA's MMA completion is multicast to both CTAs' "slot free" barrier, which gates the
//     reuse of the Delta slot two blocks later;
//   * the CTA that does not decide a block only follows the chains' state: it applies the
//     block's flips to its copy of x and of the constraint values;
//   * blocks of slack spins (past the items; W is zero there, F = 0) are decided by both CTAs
//     identically (same state, same noise), with no exchange and no MMA.
// So the two CTAs always hold identical chain states, and the decisions are those of the plain
// sampler bit for bit.  At the end CTA 1 sends its part of sum_i x_i F_i to CTA 0 through
// distributed shared memory and CTA 0 writes the outputs.
//
// Warps 0-3 decide or follow (warp w owns chains 32w..32w+31 = TMEM lanes); warps 4-7 produce
// the noise two blocks ahead, and lane 0 of warp 4 streams the W tiles.  Every wait is bounded
// (on expiry: SAIS_ETIMEOUT, stop, drain, free TMEM); every thread of both CTAs reaches the two
// cluster barriers (after initialisation, before the final readout).
#include "sais_device.cuh"
#include "sais_tc.cuh"

namespace sais {
namespace {

constexpr int kPK = 16;                 // spins per block
constexpr int kPLanes = 128;            // chains per CTA pair
constexpr int kPThreads = 256;
constexpr int kPNoiseWarp0 = 4;
constexpr uint32_t kPRing = 3;          // W tile slots
constexpr long long kPWaitCycles = 8000000000ll;
constexpr uint32_t kASlotBytes = kPLanes * kPK * 2;   // 4096
constexpr uint32_t kASlots = 4;                       // Delta ring: a decider runs 3 blocks ahead

// bars: 0 never completed (timeout test), 1 own MMAs done (one phase per item block),
// 2..5 Delta slot free (2 arrivals: both CTAs' MMAs), 6..9 Delta slot filled by the peer
// (this CTA arms it with the expected 4096 bytes; the peer's asynchronous stores complete
// them), 10..13 drain, 14..21 noise full (2 q + slot),
// 22..29 noise consumed, 30..32 tile full, 33..35 tile free, 36..37 (CTA 0) CTA 1's partial
// cost of a sweep end arrived (4 arrivals: CTA 1's decision warps), 38..39 (CTA 1) that slot
// read by CTA 0 (4 arrivals).  The last two pairs serve the best-in-run option only.
constexpr int kBars = 40;
constexpr int kBarMma = 1, kBarFree = 2, kBarFull = 6, kBarDrain = 10, kBarNoise = 14,
              kBarNoiseFree = 22, kBarTile = 30, kBarTileFree = 33, kBarCost = 36,
              kBarCostFree = 38;

__device__ __forceinline__ bool p_expired(long long n, long long polls, unsigned long long t0) {
    return polls > 0 ? n >= polls : (long long)(clock64() - t0) > kPWaitCycles;
}

template <bool kCluster>
__device__ __forceinline__ bool p_wait_warp(uint64_t *bar, uint32_t parity,
                                            volatile int *abort_flag, int32_t *status,
                                            long long polls) {
    auto tw = [&]() {
        return kCluster ? tc::mbar_try_wait_cluster(bar, parity) : tc::mbar_try_wait(bar, parity);
    };
    if (__all_sync(0xffffffffu, tw())) return true;
    const unsigned long long t0 = clock64();
    for (long long n = 0;; ++n) {
        if (__all_sync(0xffffffffu, tw())) return true;
        const bool give_up = *abort_flag != 0 || p_expired(n, polls, t0);
        if (__any_sync(0xffffffffu, give_up)) {
            if ((threadIdx.x & 31) == 0 && !*abort_flag) {
                *abort_flag = 1;
                if (status) atomicExch(status, (int32_t)SAIS_ETIMEOUT);
            }
            return false;
        }
    }
}

__device__ __forceinline__ bool p_wait_one(uint64_t *bar, uint32_t parity,
                                           volatile int *abort_flag, int32_t *status) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = clock64();
    for (;;) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if (abort_flag && *abort_flag) return false;
        if ((long long)(clock64() - t0) > kPWaitCycles) {
            if (abort_flag) *abort_flag = 1;
            if (status) atomicExch(status, (int32_t)SAIS_ETIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ uint32_t p_bf16_pm1(int d) {
    return d > 0 ? 0x3F80u : (d < 0 ? 0xBF80u : 0u);
}
// Flip of a BF16 -1/0/+1 code.
__device__ __forceinline__ int p_code(uint32_t h) { return h == 0x3F80u ? 1 : (h == 0xBF80u ? -1 : 0); }

// Item columns of the pair: n_pad = n rounded up to 16, CTA 0 holds [0, h), CTA 1 [h, n_pad),
// h = n_pad / 2 rounded up to 16 (so every MMA's N is a multiple of 16).  When h + 8 <= 512
// columns (n <= 992) each CTA's TMEM also holds 8 columns for the A operand of its own MMAs (the
// flips of a block it decides, two BF16 per column); above that the A operand of those MMAs is
// the shared-memory Delta slot, written by generic stores behind a proxy fence.
__host__ __device__ inline int pair_npad(int n) { return (n + 15) / 16 * 16; }
__host__ __device__ inline int pair_half(int npi) { return ((npi / 2) + 15) / 16 * 16; }
__host__ __device__ inline bool pair_a_in_tmem(int max_n) { return pair_half(pair_npad(max_n)) + 8 <= 512; }

template <int MC, bool kHiLo>
__global__ void __launch_bounds__(kPThreads, 1)
    pair_sampler_kernel(SampleArgs a, int32_t *status, long long polls, uint32_t tmem_cols,
                        uint32_t slot_cap, int a_tmem) {
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int kPreM = MC < 2 ? MC : 2;
    const uint32_t rank = tc::cluster_ctarank(), peer = rank ^ 1u;
    const int pair_id = blockIdx.x >> 1;
    const int j = a.work ? a.work[2 * pair_id] : (int)blockIdx.y;
    const int grp = a.work ? a.work[2 * pair_id + 1] : pair_id;
    const InstDev *__restrict__ ip = a.inst + j;
    const int m = ip->m, nprime = ip->nprime, npad = ip->npad, words = ip->words;
    const int npi = pair_npad(ip->n), h = pair_half(npi);
    const int col0 = rank == 0 ? 0 : h, ncol = rank == 0 ? h : npi - h;
    const int nb = (nprime + kPK - 1) / kPK;      // blocks per sweep
    const int nbi = min(npi / kPK, nb);           // item blocks per sweep (they come first)
    const int split_b = h / kPK;                  // item blocks [0, split_b) belong to CTA 0
    const uint32_t tile_bytes = 2u * (uint32_t)ncol * 16u;   // one term: 2 chunks x ncol rows
    const uint32_t slot_bytes = tile_bytes * (kHiLo ? 2u : 1u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    unsigned char *ring = smem;                                       // kPRing x slot_cap
    unsigned char *aslot = smem + kPRing * slot_cap;                  // kASlots x 4096
    uint32_t *xs = reinterpret_cast<uint32_t *>(aslot + kASlots * kASlotBytes);
    float *thbuf = reinterpret_cast<float *>(xs + words * kPLanes);   // [2][K][128]
    long long *part = reinterpret_cast<long long *>(thbuf + 2 * kPK * kPLanes);   // [2][128]
    long long *cpart = part + 2 * kPLanes;   // [2][128] CTA 1's partial costs at sweep ends
    long long *rbest_s = cpart + 2 * kPLanes;                                     // [128]
    int32_t *rinfo_s = reinterpret_cast<int32_t *>(rbest_s + kPLanes);           // [128][2]
    int32_t *gout = rinfo_s + 2 * kPLanes;                                        // [128][8]
    uint64_t *bars = reinterpret_cast<uint64_t *>(gout + kPLanes * kMaxBlockedConstraints);
    uint32_t *arrivals = reinterpret_cast<uint32_t *>(bars + kBars);
    uint32_t *tmem_slot = arrivals + kASlots;   // arrivals: [kASlots] decision warps done
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int *warp_ok = const_cast<int *>(abort_flag) + 1;                             // [4]

    if (threadIdx.x == kPLanes) {
        for (int i = 0; i < kBars; ++i) {
            const uint32_t cnt = (i >= kBarFree && i < kBarFree + (int)kASlots) ? 2u
                                 : i >= kBarCost                                ? 4u
                                                                                : 1u;
            tc::mbar_init(&bars[i], cnt);
        }
        for (uint32_t i = 0; i < kASlots; ++i) arrivals[i] = 0u;
        *abort_flag = 0;
        tc::fence_mbar_init();
        tc::fence_proxy_async_smem();
    }
    __syncthreads();
    // Both CTAs' barriers exist before either signals the other.  TMEM is taken only after
    // this barrier and given back before the final one, so a CTA never holds TMEM while it
    // waits for its peer at a cluster barrier.
    tc::cluster_sync();
    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, tmem_cols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t iter = a.iter_dev ? *a.iter_dev : a.iter;

    if (warp >= kPNoiseWarp0) {
        const int q = warp - kPNoiseWarp0;
        const int r = q * 32 + lane;
        const uint32_t chain = (uint32_t)(grp * kPLanes + r);
        const uint64_t seed = a.seed + (uint64_t)j;
        const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
        const uint32_t total = (uint32_t)a.sweeps * (uint32_t)nb;
        uint32_t tiles = 0;   // item blocks whose tile was issued
        for (uint32_t it = 0; it < total; ++it) {
            const uint32_t slot = it & 1u;
            if (it >= 2 && !p_wait_warp<false>(&bars[kBarNoiseFree + 2 * q + slot], ((it >> 1) + 1u) & 1u,
                                               abort_flag, status, 0))
                break;
            const uint32_t t = it / (uint32_t)nb;
            const int b = (int)(it % (uint32_t)nb);
            const int s0 = b * kPK;
            if (q == 0 && b < nbi) {
                // W tile of this item block: rows [col0, col0 + ncol) of the block's two column
                // chunks (and of the lo image), into ring slot ib % 3 once its previous use is
                // done (this CTA's MMAs of item block ib - 3).
                bool okt = true;
                const uint32_t ib = t * (uint32_t)nbi + (uint32_t)b;
                if (lane == 0) {
                    const uint32_t ts = ib % kPRing;
                    if (ib >= kPRing)
                        okt = p_wait_one(&bars[kBarTileFree + ts], ((ib / kPRing) - 1u) & 1u, abort_flag,
                                         status);
                    if (okt) {
                        unsigned char *dst = ring + ts * slot_cap;
                        tc::mbar_expect_tx(&bars[kBarTile + ts], slot_bytes);
#pragma unroll
                        for (int term = 0; term < (kHiLo ? 2 : 1); ++term) {
                            const unsigned char *src = reinterpret_cast<const unsigned char *>(
                                term ? ip->Wbf_lo : ip->Wbf);
#pragma unroll
                            for (int c = 0; c < 2; ++c)
                                tc::bulk_g2s(dst + term * tile_bytes + (uint32_t)c * ncol * 16u,
                                             src + ((size_t)((s0 >> 3) + c) * npad + col0) * 16,
                                             (uint32_t)ncol * 16u, &bars[kBarTile + ts]);
                        }
                        ++tiles;
                    }
                }
                if (__shfl_sync(0xffffffffu, okt ? 1 : 0, 0) == 0) break;
            }
            float *tb = thbuf + slot * kPK * kPLanes;
#pragma unroll
            for (int g4 = 0; g4 < kPK / 4; ++g4) {
                const uint4 rw = philox4x32_10(
                    make_uint4((uint32_t)((s0 >> 2) + g4), t, chain, iter), key0, key1);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const bool real = s0 + 4 * g4 + e < nprime;
                    tb[(4 * g4 + e) * kPLanes + r] = real ? theta_of_word(word_of(rw, e)) : -1e30f;
                }
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&bars[kBarNoise + 2 * q + slot]);
        }
        if (q == 0 && lane == 0) {
            for (uint32_t ts = 0; ts < kPRing && ts < tiles; ++ts) {
                const uint32_t uses = (tiles - ts + kPRing - 1u) / kPRing;
                p_wait_one(&bars[kBarTile + ts], (uses - 1u) & 1u, nullptr, status);
            }
        }
        __syncwarp();
    } else {
        const int r = threadIdx.x;
        const int chain = grp * kPLanes + r;
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
        const uint32_t a_own = tc::smem_u32(aslot);
        const uint32_t a_peer = tc::mapa(a_own, peer);
        const uint32_t rowoff = (uint32_t)((r >> 3) * 128 + (r & 7) * 16);   // K-major A row

        for (int w = 0; w < words; ++w) xs[w * kPLanes + r] = 0u;
        for (int c0 = 0; c0 < ncol; c0 += 32) {
            if (c0 + 32 <= ncol) {
                float v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = __ldg(hF + col0 + c0 + i);
                tc::tmem_st32(lane_addr + (uint32_t)c0, v);
            } else {   // a 16-column tail
#pragma unroll
                for (int h8 = 0; h8 < 2; ++h8) {
                    uint32_t v8[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) v8[i] = __float_as_uint(__ldg(hF + col0 + c0 + 8 * h8 + i));
                    tc::tmem_st8(lane_addr + (uint32_t)(c0 + 8 * h8), v8);
                }
            }
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
        // Constraint values as FP32 too (exact: |g| < 2^24), updated on the decision chain without
        // conversions; the int32 copy is refreshed where needed (exact re-runs, readout).
        float gf[MC];
#pragma unroll
        for (int k = 0; k < MC; ++k) gf[k] = (float)g[k];
        const float errk = field_err_factor(m);
        bool ok = polls > 0 ? p_wait_warp<false>(&bars[0], 0, abort_flag, status, polls) : true;
        uint32_t it = 0, ib = 0, cons_par = 0u;   // bit s: parity of Delta slot s's next fill
        float th[kPK];
        // Best feasible sweep-end state of the run (a.run_cost set).  Both CTAs hold the same
        // chain states, so both see which chains are feasible at a sweep end; where a chain of
        // the warp is, each CTA reads sum_i x_i F_i over its own item columns off TMEM (after
        // its last MMA of the sweep), CTA 1 sends its part to CTA 0, and CTA 0 forms the cost
        // -(sum_i x_i F_i + h^T x)/2 and keeps the best.  The block path is untouched.
        const bool track = a.run_cost != nullptr;
        long long rbest = LLONG_MAX;
        int rsweep = -1, rnf = 0;
        for (int t = 0; ok && t < a.sweeps; ++t) {
            const float beta = beta_of_sweep(a.beta_max, t, a.sweeps);
            const float hb = 0.5f * beta;
            const float ez = hb * errk;
            for (int b = 0; b < nb; ++b) {
                const int s0 = b * kPK;
                const bool item = b < nbi;
                const int owner = !item ? 2 : (b < split_b ? 0 : 1);
                const bool decide = owner == 2 || owner == (int)rank;
                const uint32_t slot = it & 1u;
                if (!p_wait_warp<false>(&bars[kBarNoise + 2 * warp + slot], (it >> 1) & 1u, abort_flag,
                                        status, polls)) {
                    ok = false;
                    break;
                }
                if (decide) {
#pragma unroll
                    for (int ii = 0; ii < kPK; ++ii) th[ii] = thbuf[(slot * kPK + ii) * kPLanes + r];
                }
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&bars[kBarNoiseFree + 2 * warp + slot]);
                const uint32_t ts = ib % kPRing;
                const unsigned char *wblk = ring + ts * slot_cap;
                if (item && !p_wait_warp<false>(&bars[kBarTile + ts], (ib / kPRing) & 1u, abort_flag,
                                                status, polls)) {
                    ok = false;
                    break;
                }
                const int wi = s0 >> 5, sb = s0 & 31;
                uint32_t xw = xs[wi * kPLanes + r];
                const uint32_t xold = xw;
                const uint32_t as = ib % kASlots;   // Delta slot of this item block
                // At every item block both CTAs wait for (a) their own MMAs of block ib - 1 (MMAs
                // complete in issue order, so all earlier ones too) and (b) the Delta slot's
                // previous use (block ib - 4) done by both CTAs' MMAs: the owner before
                // overwriting it, the follower so that it observes every phase of both barriers
                // in order (a parity wait needs that).
                // Per-spin constants of the block, loaded together (independent loads, ahead of
                // the waits below, which they overlap) for the decisions or for following the
                // peer's flips.
                float Dp[kPK], Sp[kPK];
                float Ap[kPK][kPreM];
#pragma unroll
                for (int ii = 0; ii < kPK; ++ii) {
                    const float4 sc = __ldg(ip->spinc + s0 + ii);
                    Ap[ii][0] = sc.x;
                    Dp[ii] = sc.y;
                    Sp[ii] = sc.z;
                    if (kPreM > 1) Ap[ii][kPreM > 1 ? 1 : 0] = sc.w;
                }
                if (item && ib >= 1 &&
                    (!p_wait_warp<false>(&bars[kBarMma], (ib - 1u) & 1u, abort_flag, status, polls) ||
                     (ib >= kASlots &&
                      !p_wait_warp<true>(&bars[kBarFree + as], ((ib - kASlots) / kASlots) & 1u,
                                         abort_flag, status, polls)))) {
                    ok = false;
                    break;
                }
                uint4 dlo = make_uint4(0u, 0u, 0u, 0u), dhi = dlo;
                bool send = false;
                if (decide) {
                    float Fr[kPK];
                    if (item) {
                        if (ib > 0) tc::tc_fence_after();
                        tc::tmem_ld16(lane_addr + (uint32_t)(s0 - col0), Fr);
                    } else {
#pragma unroll
                        for (int ii = 0; ii < kPK; ++ii) Fr[ii] = 0.f;   // slack spins: F = 0
                    }
                    float gf0[MC], cb[MC];
                    const float M0 = Mmax;
#pragma unroll
                    for (int k = 0; k < MC; ++k) {
                        gf0[k] = gf[k];
                        cb[k] = c[k];
                    }
                    bool near_tie = false;
#pragma unroll
                    for (int ii = 0; ii < kPK; ++ii) {
                        const int s = s0 + ii;
                        uint4 wrow[2], wrlo[2];
                        if (item) {
#pragma unroll
                            for (int cc = (ii + 1) >> 3; cc < 2; ++cc) {
                                const size_t off = ((size_t)cc * ncol + (s - col0)) * 16;
                                wrow[cc] = *reinterpret_cast<const uint4 *>(wblk + off);
                                if (kHiLo)
                                    wrlo[cc] = *reinterpret_cast<const uint4 *>(wblk + tile_bytes + off);
                            }
                        }
                        const float Fi = Fr[ii];
                        // Spin ii's bit is unchanged since the block started: read from the block-start word,
                        // so that it does not wait on the earlier flips.  The +-D_i term goes into the first
                        // product (one rounding and one dependent operation fewer; the error bound holds).
                        const int xi = (xold >> (sb + ii)) & 1;
                        float akf[MC];
                        const float Di = Dp[ii];
                        float acc = fmaf(sf, Fi, xi ? Di : -Di);
                        const float tabs = fabsf(sf * Fi);
#pragma unroll
                        for (int k = 0; k < MC; ++k) {
                            if (k < kPreM)
                                akf[k] = Ap[ii][k < kPreM ? k : 0];
                            else
                                akf[k] = (k < m) ? (float)__ldg(acol + (size_t)s * m + k) : 0.f;
                            acc = fmaf(-akf[k], c[k], acc);
                        }
                        const float theta = th[ii];
                        const float y = fmaf(hb, acc, theta);
                        const float bound = ez * (tabs + Sp[ii] * Mmax + Di) +
                                            kThetaRelErr * fabsf(theta) + kThetaAbsErr;
                        near_tie |= !(fabsf(y) > bound);
                        const float df = (y > 0.f ? 1.f : 0.f) - (xi ? 1.f : 0.f);
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
                        if (item && ii + 1 < kPK) {
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
                                float w = half(wrow[jj >> 3], jj & 7);
                                if (kHiLo) w += half(wrlo[jj >> 3], jj & 7);   // exact: integers
                                return w;
                            };
                            Fr[ii + 1] = fmaf(df, wcol(ii + 1), Fr[ii + 1]);
                            if (ii + 2 < kPK && __any_sync(0xffffffffu, df != 0.f)) {
#pragma unroll
                                for (int jj = ii + 2; jj < kPK; ++jj)
                                    Fr[jj] = fmaf(df, wcol(jj), Fr[jj]);
                            }
                        }
                    }
                    if (__any_sync(0xffffffffu, near_tie)) {
                        // Exact re-run of the block from its start state (see the single-CTA
                        // sampler): F from TMEM plus the block's earlier flips, FP64 where the
                        // FP32 bound cannot settle the decision.
                        xw = xold;
                        Mmax = M0;
#pragma unroll
                        for (int k = 0; k < MC; ++k) {
                            g[k] = (int32_t)gf0[k];
                            c[k] = cb[k];
                        }
#pragma unroll 1
                        for (int ii = 0; ii < kPK; ++ii) {
                            const int s = s0 + ii;
                            float Fi = 0.f;
                            if (item) {
                                uint32_t fv;
                                asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                                             : "=r"(fv)
                                             : "r"(lane_addr + (uint32_t)(s - col0)));
                                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                                Fi = __uint_as_float(fv);
                                uint32_t fl = ((xw ^ xold) >> sb) & ((1u << ii) - 1u);
                                while (fl) {
                                    const int i2 = __ffs(fl) - 1;
                                    fl &= fl - 1u;
                                    const int d2 = (int)((xw >> (sb + i2)) & 1u) -
                                                   (int)((xold >> (sb + i2)) & 1u);
                                    const size_t off =
                                        ((size_t)(i2 >> 3) * ncol + (s - col0)) * 16 + (i2 & 7) * 2;
                                    float w = __uint_as_float(
                                        (uint32_t)*reinterpret_cast<const uint16_t *>(wblk + off) << 16);
                                    if (kHiLo)
                                        w += __uint_as_float(
                                            (uint32_t)*reinterpret_cast<const uint16_t *>(
                                                wblk + tile_bytes + off)
                                            << 16);
                                    Fi = fmaf((float)d2, w, Fi);
                                }
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
                            const float theta = s < nprime ? theta_of_word(word_of(rw, s & 3)) : -1e30f;
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
                    xs[wi * kPLanes + r] = xw;
                    if (item) {
                        // Delta into this CTA's slot and the peer's (distributed shared memory).
                        uint32_t pk[8];
#pragma unroll
                        for (int e2 = 0; e2 < 8; ++e2) {
                            const int i0 = sb + 2 * e2;
                            const int d0 = (int)((xw >> i0) & 1u) - (int)((xold >> i0) & 1u);
                            const int d1 = (int)((xw >> (i0 + 1)) & 1u) - (int)((xold >> (i0 + 1)) & 1u);
                            pk[e2] = p_bf16_pm1(d0) | (p_bf16_pm1(d1) << 16);
                        }
                        const uint4 lo4 = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        const uint4 hi4 = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                        // This CTA's MMA takes the flips from TMEM (8 columns after F; the
                        // previous block's MMAs, which read them, are done): no shared-memory
                        // write and no proxy fence on this path.  Without room in TMEM, from
                        // this CTA's Delta slot behind a proxy fence.  The peer's copy goes out
                        // after this CTA's MMAs are issued (below).
                        if (a_tmem) {
                            tc::tmem_st8(lane_addr + (uint32_t)ncol, pk);
                            tc::tc_fence_before();
                        } else {
                            const uint32_t off = as * kASlotBytes + rowoff;
                            *reinterpret_cast<uint4 *>(aslot + off) = lo4;
                            *reinterpret_cast<uint4 *>(aslot + off + 2048) = hi4;
                            tc::fence_proxy_async_smem();
                        }
                        dlo = lo4;
                        dhi = hi4;
                        send = true;
                    }
                } else {
                    // The peer decides this block: take its flips from the Delta slot.
                    const uint32_t ph = (cons_par >> as) & 1u;
                    if (warp == 0 && lane == 0) tc::mbar_expect_tx(&bars[kBarFull + as], kASlotBytes);
                    if (!p_wait_warp<true>(&bars[kBarFull + as], ph, abort_flag, status, polls)) {
                        ok = false;
                        break;
                    }
                    cons_par ^= 1u << as;
                    const uint32_t off = as * kASlotBytes + rowoff;
                    const uint4 lo4 = *reinterpret_cast<const uint4 *>(aslot + off);
                    const uint4 hi4 = *reinterpret_cast<const uint4 *>(aslot + off + 2048);
                    const uint32_t pk[8] = {lo4.x, lo4.y, lo4.z, lo4.w, hi4.x, hi4.y, hi4.z, hi4.w};
#pragma unroll
                    for (int ii = 0; ii < kPK; ++ii) {
                        const int d = p_code((pk[ii >> 1] >> ((ii & 1) * 16)) & 0xFFFFu);
                        xw ^= (uint32_t)(d != 0) << (sb + ii);
#pragma unroll
                        for (int k = 0; k < MC; ++k) {
                            if (k < kPreM)
                                gf[k] = fmaf(Ap[ii][k < kPreM ? k : 0], (float)d, gf[k]);
                            else if (k < m && d != 0)
                                gf[k] = fmaf((float)__ldg(acol + (size_t)(s0 + ii) * m + k),
                                             (float)d, gf[k]);
                        }
                    }
                    Mmax = 0.f;
#pragma unroll
                    for (int k = 0; k < MC; ++k) {
                        if (k < m) {
                            c[k] = fmaf(kappa, gf[k], cA[k]);
                            Mmax = fmaxf(Mmax, fmaf(fabsf(kappa), fabsf(gf[k]), fabsf(cA[k])));
                        }
                    }
                    xs[wi * kPLanes + r] = xw;
                    __syncwarp();
                }
                if (item) {
                    // The last of the four decision warps issues this CTA's MMAs for the block:
                    // F[:, half] += W[half, blk] Delta[blk, :], A = the Delta slot (K-major,
                    // LBO 2048, SBO 128), B = the W tile (LBO 16 ncol, SBO 128).
                    if (lane == 0) {
                        __threadfence_block();
                        const bool last = (atomicAdd(&arrivals[as], 1u) & 3u) == 3u;
                        if (last) {
                            __threadfence_block();
                            if (send && !a_tmem) tc::fence_proxy_async_smem();
                            tc::tc_fence_after();
                            const uint32_t lbo_b = (uint32_t)ncol * 16u;
                            const uint32_t w_base = tc::smem_u32(wblk);
                            const uint64_t adesc = tc::smem_desc(a_own + as * kASlotBytes, 2048u, 128u);
                            auto mma_cols = [&](int c0, int c1) {
#pragma unroll
                                for (int term = 0; term < (kHiLo ? 2 : 1); ++term) {
                                    for (int j0 = c0; j0 < c1; j0 += 256) {
                                        const int nr = min(256, c1 - j0);
                                        const uint64_t bd = tc::smem_desc(
                                            w_base + (uint32_t)term * tile_bytes + (uint32_t)j0 * 16u,
                                            lbo_b, 128u);
                                        const uint32_t id = tc::idesc_bf16_f32(128, (uint32_t)nr);
                                        if (send && a_tmem)   // this CTA decided: A in TMEM
                                            tc::mma_bf16_tmem_a(tmem + (uint32_t)j0,
                                                                tmem + (uint32_t)ncol, bd, id, 1u);
                                        else   // A in the Delta slot
                                            tc::mma_bf16(tmem + (uint32_t)j0, adesc, bd, id, 1u);
                                    }
                                }
                            };
                            mma_cols(0, ncol);
                            tc::mma_commit(&bars[kBarMma]);
                            tc::mma_commit(&bars[kBarTileFree + ts]);
                            tc::mma_commit_multicast(&bars[kBarFree + as], (uint16_t)0x3u);
                        }
                    }
                    __syncwarp();
                    if (send) {
                        // Delta into the peer's slot (distributed shared memory) by asynchronous
                        // stores whose bytes complete the peer's slot-filled barrier; after this
                        // CTA's MMAs are issued, and without a fence on this CTA's path.
                        const uint32_t off = as * kASlotBytes + rowoff;
                        const uint32_t pbar = tc::mapa(tc::smem_u32(&bars[kBarFull + as]), peer);
                        tc::st_async_v4(a_peer + off, dlo, pbar);
                        tc::st_async_v4(a_peer + off + 2048, dhi, pbar);
                    }
                    ++ib;
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
                            if ((xs[(s >> 5) * kPLanes + r] >> (s & 31)) & 1u) sv += 1LL << (s - o0);
                        if ((long long)gf[k] - sv > (long long)ip->fmargin[k]) feas = false;
                    }
                }
                // This CTA's sum_i x_i F_i over its item columns, where the warp needs it.
                long long part_own = 0;
                if (__any_sync(0xffffffffu, feas)) {
                    // The sweep's last MMA of this CTA (item block ib - 1) done: F is current.
                    if (!p_wait_warp<false>(&bars[kBarMma], (ib - 1u) & 1u, abort_flag, status, polls)) {
                        ok = false;
                    } else {
                        tc::tc_fence_after();
                        for (int c0 = 0; c0 < ncol; c0 += 16) {
                            float v[16];
                            tc::tmem_ld16(lane_addr + (uint32_t)c0, v);
                            const int sc = col0 + c0;   // a multiple of 16
                            const uint32_t bits =
                                sc < words * 32 ? (xs[(sc >> 5) * kPLanes + r] >> (sc & 31)) & 0xFFFFu : 0u;
                            int32_t pf = 0;   // |F| < 2^24: 16 terms fit int32
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                if ((bits >> i) & 1u) pf += __float2int_rz(v[i]);
                            part_own += pf;
                        }
                    }
                }
                // Sweep end: CTA 1's part into CTA 0's slot t % 2 (plain stores, then a release
                // arrival), once CTA 0 has read what the slot held two sweeps ago.  Sent every
                // sweep (0 where not needed) so that both CTAs step the slots' phases together.
                const uint32_t cs = (uint32_t)t & 1u, cu = (uint32_t)t >> 1;
                if (!ok) {
                } else if (rank == 1) {
                    if (t >= 2 && !p_wait_warp<true>(&bars[kBarCostFree + cs], (cu - 1u) & 1u,
                                                     abort_flag, status, polls))
                        ok = false;
                    if (ok) {
                        tc::st_cluster_s64(tc::mapa(tc::smem_u32(cpart + cs * kPLanes + r), 0u),
                                           part_own);
                        __syncwarp();
                        if (lane == 0) {
                            tc::fence_acq_rel_cluster();
                            tc::mbar_arrive_remote(tc::mapa(tc::smem_u32(&bars[kBarCost + cs]), 0u));
                        }
                    }
                } else if (!p_wait_warp<true>(&bars[kBarCost + cs], cu & 1u, abort_flag, status,
                                              polls)) {
                    ok = false;
                } else {
                    const long long tot = part_own + cpart[cs * kPLanes + r];
                    __syncwarp();
                    if (lane == 0)
                        tc::mbar_arrive_remote(tc::mapa(tc::smem_u32(&bars[kBarCostFree + cs]), 1u));
                    if (feas) {
                        long long sumh = 0;
                        for (int w = 0; w < words; ++w) {
                            uint32_t bits = xs[w * kPLanes + r];
                            while (bits) {
                                const int i = w * 32 + __ffs(bits) - 1;
                                bits &= bits - 1u;
                                sumh += (long long)__float2int_rz(__ldg(ip->hF + i));
                            }
                        }
                        const long long cost = -(tot + sumh) / 2;
                        ++rnf;
                        if (cost < rbest) {
                            rbest = cost;
                            rsweep = t;
                            if (valid) {
                                uint32_t *rx = a.run_x + ((size_t)j * a.chains + chain) * a.words;
                                for (int w = 0; w < a.words; ++w)
                                    rx[w] = w < words ? xs[w * kPLanes + r] : 0u;
                            }
                        }
                    }
                }
            }
            if (ok && a.trace && valid && rank == 0) {
                uint32_t *tr = a.trace + (((size_t)j * a.chains + chain) * a.sweeps + t) * a.words;
                for (int w = 0; w < a.words; ++w) tr[w] = w < words ? xs[w * kPLanes + r] : 0u;
            }
        }
        // Drain: every MMA of this CTA completes before the readout and the TMEM release; each
        // decision warp's lane 0 commits what it issued, every warp waits for all four (bounded,
        // not cut short by an abort).
        if (lane == 0) tc::mma_commit(&bars[kBarDrain + warp]);
        __syncwarp();
        bool drained = true;
        if (lane == 0)
            for (int w = 0; w < 4; ++w)
                drained = p_wait_one(&bars[kBarDrain + w], 0, nullptr, status) && drained;
        drained = __shfl_sync(0xffffffffu, drained ? 1 : 0, 0) != 0;
        ok = ok && drained;
        tc::tc_fence_after();
        // This CTA's part of sum_i x_i F_i over its item columns, into CTA 0's part[rank][r].
        long long sumF = 0;
        if (ok) {
            for (int c0 = 0; c0 < ncol; c0 += 16) {
                float v[16];
                tc::tmem_ld16(lane_addr + (uint32_t)c0, v);
                const int s = col0 + c0;   // a multiple of 16
                const uint32_t bits =
                    s < words * 32 ? (xs[(s >> 5) * kPLanes + r] >> (s & 31)) & 0xFFFFu : 0u;
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if ((bits >> i) & 1u) sumF += (long long)v[i];
            }
        }
        if (rank == 1)
            tc::st_cluster_s64(tc::mapa(tc::smem_u32(part + kPLanes + r), 0u), sumF);
        else
            part[r] = sumF;
#pragma unroll
        for (int k = 0; k < MC; ++k) gout[r * kMaxBlockedConstraints + k] = (int32_t)gf[k];
        if (rank == 0 && track) {
            rbest_s[r] = rbest;
            rinfo_s[2 * r] = rsweep;
            rinfo_s[2 * r + 1] = rnf;
        }
        if (lane == 0) warp_ok[warp] = ok ? 1 : 0;
        __syncwarp();
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, tmem_cols);
    }
    // CTA 1's partial sums have landed in CTA 0; no remote access follows this barrier.
    tc::cluster_sync();
    // Readout of the last sample by CTA 0: cost -(sum_i x_i F_i + h^T x)/2, g, feasibility.
    if (rank == 0 && warp < kPNoiseWarp0 && warp_ok[warp] && !*abort_flag) {
        const int r = threadIdx.x;
        const int chain = grp * kPLanes + r;
        if (chain < (a.inst_chains ? a.inst_chains[j] : a.chains)) {
            long long sumh = 0;
            for (int w = 0; w < words; ++w) {
                uint32_t bits = xs[w * kPLanes + r];
                while (bits) {
                    const int i = w * 32 + __ffs(bits) - 1;
                    bits &= bits - 1u;
                    sumh += (long long)__ldg(ip->hF + i);
                }
            }
            const long long total = part[r] + part[kPLanes + r];
            const size_t cidx = (size_t)j * a.chains + chain;
            for (int w = 0; w < a.words; ++w)
                a.x[cidx * a.words + w] = w < words ? xs[w * kPLanes + r] : 0u;
            a.cost[cidx] = -(total + sumh) / 2;
            bool feas = true;
            for (int k = 0; k < m; ++k) {
                const int o0 = ip->slack_off[k], o1 = ip->slack_off[k + 1];
                long long sv = 0;
                for (int s = o0; s < o1; ++s)
                    if ((xs[(s >> 5) * kPLanes + r] >> (s & 31)) & 1u) sv += 1LL << (s - o0);
                const int32_t gk = gout[r * kMaxBlockedConstraints + k];
                if ((long long)gk - sv > (long long)ip->fmargin[k]) feas = false;
                a.g[cidx * a.m_stride + k] = gk;
            }
            for (int k = m; k < a.m_stride; ++k) a.g[cidx * a.m_stride + k] = 0;
            if (a.feasible) a.feasible[cidx] = feas ? 1 : 0;
            if (a.run_cost) {
                a.run_cost[cidx] = rbest_s[r];
                if (a.run_sweep) a.run_sweep[cidx] = rinfo_s[2 * r];
                if (a.run_nfeas) a.run_nfeas[cidx] = rinfo_s[2 * r + 1];
                if (rinfo_s[2 * r] < 0)
                    for (int w = 0; w < a.words; ++w) a.run_x[cidx * a.words + w] = 0u;
            }
        }
    }
}

}  // namespace
}  // namespace sais

namespace sais {

bool pair_eligible(int n, int m, bool has_w) {
    const int npi = pair_npad(n);
    return has_w && m <= kMaxBlockedConstraints && npi >= 128 && npi <= 1024;
}

bool pair_a_tmem(int n) { return pair_a_in_tmem(n); }

size_t pair_smem_bytes(int max_n, int max_words, bool hilo) {
    const size_t half = (size_t)pair_half(pair_npad(max_n));
    const size_t slot = 2 * half * 16 * (hilo ? 2 : 1);
    return kPRing * slot + kASlots * kASlotBytes + (size_t)max_words * kPLanes * 4 +
           (size_t)2 * kPK * kPLanes * 4 + (size_t)6 * kPLanes * 8 +
           (size_t)kPLanes * kMaxBlockedConstraints * 4 + kBars * 8 + 64;
}

namespace {
template <int MC, bool H>
cudaError_t pair_launch(const SampleArgs &a, int32_t *status, long long polls, size_t smem,
                        uint32_t cols, uint32_t slot_cap, int a_tmem, cudaStream_t st) {
    auto kern = pair_sampler_kernel<MC, H>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = a.work ? dim3(2 * a.nwork, 1) : dim3(2 * ((a.chains + kPLanes - 1) / kPLanes), a.count);
    cfg.blockDim = dim3(kPThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, a, status, polls, cols, slot_cap, a_tmem);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}
template <bool H>
cudaError_t pair_mc(const SampleArgs &a, int max_m, int32_t *status, long long polls, size_t smem,
                    uint32_t cols, uint32_t slot_cap, int at, cudaStream_t st) {
    if (max_m <= 1) return pair_launch<1, H>(a, status, polls, smem, cols, slot_cap, at, st);
    if (max_m <= 2) return pair_launch<2, H>(a, status, polls, smem, cols, slot_cap, at, st);
    if (max_m <= 4) return pair_launch<4, H>(a, status, polls, smem, cols, slot_cap, at, st);
    return pair_launch<8, H>(a, status, polls, smem, cols, slot_cap, at, st);
}
}  // namespace

cudaError_t launch_pair_sampler(const SampleArgs &a, int max_m, int max_n, int max_words, bool hilo,
                                int32_t *status, long long dec_wait_polls, cudaStream_t st) {
    const int half = pair_half(pair_npad(max_n));
    const bool a_tmem = pair_a_in_tmem(max_n);
    uint32_t cols = 32;
    while (cols < (uint32_t)half + (a_tmem ? 8u : 0u)) cols <<= 1;   // F, then the own A operand
    const uint32_t slot_cap = (uint32_t)(2 * half * 16 * (hilo ? 2 : 1));
    // one CTA per SM (its TMEM allocation may take all 512 columns)
    size_t smem = pair_smem_bytes(max_n, max_words, hilo);
    const size_t floor_smem = 228 * 1024 / 2 + 1;
    if (smem < floor_smem) smem = floor_smem;
    const long long polls = dec_wait_polls > 0 ? dec_wait_polls : 0;
    const int at = a_tmem ? 1 : 0;
    if (hilo) return pair_mc<true>(a, max_m, status, polls, smem, cols, slot_cap, at, st);
    return pair_mc<false>(a, max_m, status, polls, smem, cols, slot_cap, at, st);
}

}  // namespace sais
