// sais_field_kernel.cuh -- block-field p-bit sampler: the fields of each block of K spins come
// from one tensor-core GEMM over the current chain states.
//
// The Gibbs sweep of Sec. III-B stays sequential: spins are visited in index order and each
// decision sees every earlier flip.  The objective part of the p-bit input (Eq. 9) is the
// integer field F_i = h_i + sum_j W_ij x_j.  Spins are taken in blocks of K:
//   1. before block b, its K fields are computed from the chain states as they stand,
//      F[chains, blk] = h[blk] + X[chains, :] W[:, blk], one tcgen05.mma chain of
//      ceil(n/16) steps (M = 128 chains, N = K, K-dim = 16 item spins per step) in BF16 with
//      FP32 accumulation.  Products and partial sums are integers below 2^24, so the fields are
//      exact, equal to those the plain sampler carries;
//   2. the K decisions are made one after the other on CUDA cores, each flip correcting the
//      fields of the block's later spins (W[blk, blk], exact FP32);
//   3. the block's new states go back into X (TMEM) and the next block's GEMM is issued.
// Only the item spins enter X: slack spins have no pair values (Sec. IV-A).
//
// Tensor memory per CTA is X (BF16 0/1, 8 columns per 16 item spins) plus K columns of fields,
// so an SM holds two CTAs of 128 chains when n <= 480 (K = 16): while one CTA waits for its
// GEMM the other decides, and each SM sub-partition runs two independent decision chains.  A
// sampler that kept every field F_i resident in TMEM (N' columns per 128 chains) would fit one.
//
// Layout (one CTA = 128 chains of one instance):
//   TMEM   X: lane = chain, column c holds spins 2c (low half) and 2c+1 as BF16 0 / 1.
//          D: the block's K fields (FP32) in the last K of the CTA's columns.
//   SMEM   a ring of 3 W tiles, each the K rows of one block (BF16, the K-major B operand:
//          element (i, j) at ((i/8)(n16/8) + j/8) 128 + (i%8) 16 + (j%8) 2 bytes) followed by the
//          block's K x K diagonal in FP32 for the in-block corrections; the bit-packed states;
//          a two-slot ring of noise.
//   Warps  0-3 decide (warp w owns TMEM lanes 32w..32w+31: its 32 chains); the last of them to
//          finish a block issues the next block's GEMM.  Warps 4-7 compute the noise (Philox,
//          atanh) up to two blocks ahead; lane 0 of warp 4 also streams the W tiles by bulk
//          asynchronous copies (TMA engine).  The decision warps run with 192 registers and the
//          noise warps with 64 (setmaxnreg), from the 128 per thread the CTA launches with.
//   After the last sweep a readout pass recomputes every field from the final states for the
//   cost c(x) = -(sum_i x_i F_i + h^T x)/2.  With best-in-run tracking the cost also follows
//   every flip, c' - c = -d F_i.
// Every mbarrier wait is bounded: on expiry the kernel records SAIS_ETIMEOUT, stops, drains its
// copies and MMAs, frees TMEM and exits.
#pragma once

#include "sais_device.cuh"
#include "sais_tc.cuh"

namespace sais {

// Launch shape shared by every instantiation of the block-field sampler.
struct FieldLaunch {
    size_t smem;
    uint32_t cols;       // TMEM columns of a CTA
    int32_t max_n16;     // largest n rounded up to 16 in the launch
    int32_t ring;        // W tile slots (2 or 3)
    int32_t xs_chunks;   // 16-spin state chunks kept in shared memory (beyond TMEM), at most
};

namespace {

constexpr int kFLanes = 128;
constexpr int kFThreads = 256;
constexpr int kFNoiseWarp0 = 4;
constexpr uint32_t kFXChunkBytes = 128 * 16 * 2;   // one 16-spin state chunk, 128 chains, BF16
constexpr long long kFWaitCycles = 8000000000ll;   // about 4 s at 2 GHz
// bars: 0 never completed (timeout test), 1 and 28 the GEMM of the blocks whose fields go to
// accumulator slot 0 and 1 done (one phase per block of that slot; 5 arrivals: the four noise
// warps' parts and the last decision warp's), 2..5 drain of decision warp 0..3, 6..13 noise slot
// written (2 q + slot), 14..21 noise slot consumed, 22..24 W tile slot filled, 25..27 W tile slot
// free (4 arrivals: every decision warp is done with the block); the ring uses the first L.ring
// of each; 29..32 drain of noise warp 0..3
constexpr int kFBarNever = 0, kFBarMma = 1, kFBarDrain = 2, kFBarNoise = 6, kFBarNoiseFree = 14,
              kFBarTile = 22, kFBarTileFree = 25, kFBarMma1 = 28, kFBarNDrain = 29, kFBars = 33;

__device__ __forceinline__ bool f_expired(long long n, long long polls, unsigned long long t0) {
    return polls > 0 ? n >= polls : (long long)(clock64() - t0) > kFWaitCycles;
}

__device__ __forceinline__ bool f_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                       int32_t *status, long long polls) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = clock64();
    for (long long n = 0;; ++n) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if (abort_flag && *abort_flag) return false;
        if (f_expired(n, polls, t0)) {
            if (abort_flag) *abort_flag = 1;
            if (status) atomicExch(status, (int32_t)SAIS_ETIMEOUT);
            return false;
        }
    }
}

// Warp-collective bounded wait: the warp leaves together, when every lane has seen the phase or
// when any lane sees the abort flag or the limit.
__device__ __forceinline__ bool f_wait_warp(uint64_t *bar, uint32_t parity,
                                            volatile int *abort_flag, int32_t *status,
                                            long long polls) {
    if (__all_sync(0xffffffffu, tc::mbar_try_wait(bar, parity))) return true;
    const unsigned long long t0 = clock64();
    for (long long n = 0;; ++n) {
        const bool got = tc::mbar_try_wait(bar, parity);
        if (__all_sync(0xffffffffu, got)) return true;
        const bool give_up = *abort_flag != 0 || f_expired(n, polls, t0);
        if (__any_sync(0xffffffffu, give_up)) {
            if ((threadIdx.x & 31) == 0 && !*abort_flag) {
                *abort_flag = 1;
                if (status) atomicExch(status, (int32_t)SAIS_ETIMEOUT);
            }
            return false;
        }
    }
}

// 32 lanes x K columns of the fields (warp-collective), waited for.  With the hi/lo split the
// accumulator holds the hi products in its first K columns and the lo products in the next K;
// their sum is exact (integers below 2^24).
template <int K, bool kHiLo>
__device__ __forceinline__ void f_load_fields(uint32_t taddr, float (&r)[K]) {
    if constexpr (K == 16 && kHiLo) {   // both terms in one load
        float v[32];
        tc::tmem_ld32(taddr, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) r[i] = v[i] + v[16 + i];
        return;
    } else if constexpr (K == 16) {
        tc::tmem_ld16(taddr, r);
    } else {
#pragma unroll
        for (int c = 0; c < K; c += 32) {
            float v[32];
            tc::tmem_ld32(taddr + (uint32_t)c, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) r[c + i] = v[i];
        }
    }
    if constexpr (kHiLo && K != 16) {
#pragma unroll
        for (int c = 0; c < K; c += 16) {
            float v[16];
            tc::tmem_ld16(taddr + (uint32_t)(K + c), v);
#pragma unroll
            for (int i = 0; i < 16; ++i) r[c + i] += v[i];
        }
    }
}

// Round and slot of tile u in a ring of 2 or 3 slots (a shift or a multiply-high, not a
// division by a runtime value).
__device__ __forceinline__ uint32_t f_round(uint32_t u, uint32_t ring) {
    return ring == 3u ? u / 3u : u >> 1;
}
__device__ __forceinline__ uint32_t f_slot(uint32_t u, uint32_t ring) {
    return u - f_round(u, ring) * ring;
}

template <int K>
__device__ __forceinline__ const float *f_diag_image(const InstDev *ip) {
    return K == 16 ? ip->Wdiag : (K == 32 ? ip->Wd32 : ip->Wd64);
}

// One work item: 128 chains (group `grp`) of instance j, on a CTA of 256 threads that holds
// `tmem` (L.cols columns) and dynamic shared memory sized for the launch (declared here, not
// passed as a pointer, so that every access stays a shared-memory access).  Returns
// false when a bounded wait gave up (SAIS_ETIMEOUT recorded).  kSplit: the decision / noise
// warpgroups move to 192 / 64 registers (a CTA launched with 128 per thread; once per CTA).
template <int MC, int K, bool kHiLo, bool kTrack, bool kSplit>
__device__ __forceinline__ bool field_item(const SampleArgs &a, int j, int grp, uint32_t tmem,
                                           const FieldLaunch &L, int32_t *status,
                                           long long dec_wait_polls) {
    extern __shared__ __align__(1024) unsigned char smem[];
    if (!SAIS_DCHECK(status, j >= 0 && j < a.count && grp >= 0 && grp * kFLanes < a.chains))
        return false;
    constexpr int kXW = K >= 32 ? K / 32 : 1;   // state words a block spans
    const uint32_t kFRing = (uint32_t)L.ring;
    const uint32_t tmem_cols = L.cols;
    const int32_t max_n16 = L.max_n16;
    const InstDev *__restrict__ ip = a.inst + j;
    const int m = ip->m, nprime = ip->nprime, words = ip->words, n16 = ip->n16;
    const int kx = n16 / 16;                   // GEMM steps per block
    // Accumulator columns of a block: K, or 2K with the hi/lo split, whose two W tiles lie one
    // after the other in shared memory and so form one B operand of N = 2K (an MMA costs the
    // same for any N up to 128): one GEMM computes both terms.  Two slots: block u's fields in
    // slot u & 1, so that warps done with block u can start the GEMM of block u + 1 while the
    // others still read block u's fields (the exact re-run reads them again).
    constexpr int KD = kHiLo ? 2 * K : K;
    // State chunks in TMEM (columns 8 kc); the rest in shared memory as SMEM A operands.
    const int kxt = min(kx, (int)((tmem_cols - 2u * (uint32_t)KD) / 8u));
    const int nb = (nprime + K - 1) / K;       // blocks per sweep
    const uint32_t tile_bytes = (uint32_t)K * (uint32_t)n16 * 2u;   // one BF16 term, one block
    const uint32_t diag_off = tile_bytes * (kHiLo ? 2u : 1u);
    // K >= 32: after the diagonal, the block's per-spin records {a_0i, D_i, sum_k a_ki, a_1i} and
    // h (K x 16 and K x 4 bytes), staged with the tile so that no global load waits on the
    // block's path.  (K = 16 loads them from global memory while it waits for the GEMM: measured
    // faster there, where the staging warp's extra copies cost more than they save.)
    constexpr bool kSide = K >= 32;
    const uint32_t side_off = diag_off + (uint32_t)(K * K * 4);
    const uint32_t slot_stride = (uint32_t)K * (uint32_t)max_n16 * 2u * (kHiLo ? 2u : 1u) +
                                 (uint32_t)(K * K * 4) + (kSide ? (uint32_t)(K * 20) : 0u);
    const uint32_t dcol0 = tmem_cols - 2u * (uint32_t)KD;   // the fields D: last 2 KD columns
    const uint32_t total = (uint32_t)a.sweeps * (uint32_t)nb + (uint32_t)nb;   // + readout pass
    const uint32_t ndec = (uint32_t)a.sweeps * (uint32_t)nb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // State words per chain in shared memory: an even count, since a block of K = 64 spins may
    // span one word past ceil(N'/32) (padding spins, always 0).
    const int xwords = (words + 1) & ~1;
    unsigned char *ring = smem;
    // State chunks beyond TMEM: chain c's 16 values of a chunk at (c/8) 256 + (c%8) 16 bytes
    // (spins 0-7) and 128 bytes further (spins 8-15), the no-swizzle K-major A operand (LBO 128,
    // SBO 256 bytes).
    unsigned char *xsm = smem + kFRing * slot_stride;
    uint32_t *xs = reinterpret_cast<uint32_t *>(xsm + (size_t)L.xs_chunks * kFXChunkBytes);
    float *thbuf = reinterpret_cast<float *>(xs + xwords * kFLanes);   // [2][K][128] noise
    uint64_t *bars = reinterpret_cast<uint64_t *>(thbuf + 2 * K * kFLanes);
    uint32_t *arrivals = reinterpret_cast<uint32_t *>(bars + kFBars);   // [3]
    volatile int *abort_flag = reinterpret_cast<volatile int *>(arrivals + 4);

    // Debug builds: the launch's shape against this item (the host's sizing makes these hold;
    // every thread evaluates the same values).
    if (!SAIS_DCHECK(status, n16 % 16 == 0 && n16 <= max_n16 && nb * K <= ip->npad &&
                                 8u * (uint32_t)kxt + 2u * (uint32_t)KD <= tmem_cols &&
                                 kx - kxt <= L.xs_chunks && (kFRing == 2u || kFRing == 3u) &&
                                 (uint32_t)(reinterpret_cast<unsigned char *>(
                                                const_cast<int *>(abort_flag) + 1) -
                                            smem) <= dynamic_smem_bytes()))
        return false;
    // The barriers start afresh for every item (the previous item's waits are all over).
    if (threadIdx.x == 0) {
        for (int i = 0; i < kFBars; ++i)
            tc::mbar_init(&bars[i], (i >= kFBarTileFree && i < kFBarTileFree + 3)
                                        ? 4u
                                        : ((i == kFBarMma || i == kFBarMma1) ? 5u : 1u));
        arrivals[0] = arrivals[1] = arrivals[2] = 0u;
        *abort_flag = 0;
        tc::fence_mbar_init();
        tc::fence_proxy_async_smem();
    }
    __syncthreads();
    const uint32_t iter = a.iter_dev ? *a.iter_dev : a.iter;

    // The GEMM of block v, D(v) = X [W_hi | W_lo][:, blk(v)], one MMA per 16-spin state chunk,
    // into accumulator slot v & 1, which was zeroed before: every MMA accumulates, so their order
    // does not matter (sums of exact integers below 2^24).  An MMA holds its issuing warp about as
    // long as it runs, whatever N <= 128, and warps issue in parallel.  So the GEMM is split: the
    // chunks block v - 1 leaves unchanged are issued by the four noise warps (chunks kc = q mod 4)
    // as soon as block v - 2 is done, while block v - 1 is being decided; the last decision warp
    // to finish block v - 1 adds the chunks it changed.  (v < 2: that warp issues it all.)
    const uint32_t idesc = tc::idesc_bf16_f32(128, (uint32_t)KD);
    // Chunks [c0, c1) changed by block u's decisions (none for the readout pass, or past the
    // items).
    auto changed = [&](uint32_t u, int &c0, int &c1) {
        c0 = c1 = 0;
        if (u >= ndec) return;
        const int s0u = (int)(u % (uint32_t)nb) * K;
        if (s0u >= n16) return;
        c0 = s0u >> 4;
        c1 = min(kx, c0 + K / 16);
    };
    // MMAs over chunks k0, k0 + step, ... < k1 into the slot of block v: A from TMEM for chunks
    // below kxt, then from shared memory (separate loops: no branch around an MMA).
    auto mma_chunks = [&](uint32_t v, int k0, int k1, int step) {
        const uint32_t base = tc::smem_u32(ring + f_slot(v, kFRing) * slot_stride);
        const uint32_t d = tmem + dcol0 + (v & 1u) * (uint32_t)KD;
        // B: 8-row groups every 16 n16 bytes (the lo tile, tile_bytes after the hi one, continues
        // the hi tile's row groups); chunk kc starts 256 kc bytes in (16 kc in the descriptor's
        // address field, which stays below 2^14 in shared memory).
        const uint64_t bd0 = tc::smem_desc(base, 128u, (uint32_t)n16 * 16u);
        const uint64_t ad0 = tc::smem_desc(tc::smem_u32(xsm), 128u, 256u);
        int kc = k0;
        for (; kc < min(k1, kxt); kc += step)
            tc::mma_bf16_tmem_a(d, tmem + 8u * (uint32_t)kc, bd0 + 16u * (uint32_t)kc, idesc, 1u);
        for (; kc < k1; kc += step)
            tc::mma_bf16(d, ad0 + (uint32_t)(kc - kxt) * (kFXChunkBytes >> 4),
                         bd0 + 16u * (uint32_t)kc, idesc, 1u);
    };
    auto mma_bar = [&](uint32_t v) { return &bars[(v & 1u) ? kFBarMma1 : kFBarMma]; };
    auto tile_ready = [&](uint32_t v) -> bool {
        return f_wait(&bars[kFBarTile + f_slot(v, kFRing)], f_round(v, kFRing) & 1u, abort_flag,
                      status, 0);
    };

    if (warp >= kFNoiseWarp0) {
        if (kSplit) asm volatile("setmaxnreg.dec.sync.aligned.u32 64;");
        // Noise warps: warp 4+q produces theta = atanh(rho) for the chains of decision warp q, up
        // to two blocks ahead, into a two-slot ring.  Lane 0 of warp 4 streams the W tiles.
        const int q = warp - kFNoiseWarp0;
        const int r = q * 32 + lane;
        const uint32_t chain = (uint32_t)(grp * kFLanes + r);
        const uint64_t seed = a.seed + (uint64_t)j;
        const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
        const unsigned char *Wg = reinterpret_cast<const unsigned char *>(ip->Wg);
        const unsigned char *Wgl = reinterpret_cast<const unsigned char *>(ip->Wg_lo);
        const unsigned char *Wd = reinterpret_cast<const unsigned char *>(f_diag_image<K>(ip));
        const bool stager = q == 0 && lane == 0;
        uint32_t tiles_issued = 0;
        // W tile of block u (decision or readout) into slot u % kFRing, once that slot's previous
        // block (u - kFRing) is done.
        auto stage = [&](uint32_t u) -> bool {
            const uint32_t ts = f_slot(u, kFRing);
            if (u >= kFRing &&
                !f_wait(&bars[kFBarTileFree + ts], (f_round(u, kFRing) - 1u) & 1u, abort_flag,
                        status, 0))
                return false;
            const uint32_t b = u < ndec ? u % (uint32_t)nb : u - ndec;
            unsigned char *dst = ring + ts * slot_stride;
            const uint32_t dbytes = (uint32_t)(K * K * 4);
            tc::mbar_expect_tx(&bars[kFBarTile + ts],
                               diag_off + dbytes + (kSide ? (uint32_t)(K * 20) : 0u));
            tc::bulk_g2s(dst, Wg + (size_t)b * tile_bytes, tile_bytes, &bars[kFBarTile + ts]);
            if (kHiLo)
                tc::bulk_g2s(dst + tile_bytes, Wgl + (size_t)b * tile_bytes, tile_bytes,
                             &bars[kFBarTile + ts]);
            tc::bulk_g2s(dst + diag_off, Wd + (size_t)b * dbytes, dbytes, &bars[kFBarTile + ts]);
            if (kSide) {   // (N'_pad is a multiple of 64: the block's records are in the arrays)
                tc::bulk_g2s(dst + side_off, ip->spinc + (size_t)b * K, (uint32_t)(K * 16),
                             &bars[kFBarTile + ts]);
                tc::bulk_g2s(dst + side_off + (uint32_t)(K * 16), ip->hF + (size_t)b * K,
                             (uint32_t)(K * 4), &bars[kFBarTile + ts]);
            }
            ++tiles_issued;
            return true;
        };
        // This warp's part of block v's GEMM (v >= 2): its chunks (q mod 4) that block v - 1
        // leaves unchanged, once block v - 2 is done (its X chunks written and slot v & 1 zeroed:
        // the tile-free barrier of block v - 2) and block v's tile is in; then its commit.  (v < 2:
        // the commit alone, which arrives at once.)  Lane 0.
        auto issue_ahead = [&](uint32_t v) -> bool {
            if (v >= 2u) {
                const uint32_t u = v - 2u;
                if (!f_wait(&bars[kFBarTileFree + f_slot(u, kFRing)], f_round(u, kFRing) & 1u,
                            abort_flag, status, 0) ||
                    !tile_ready(v))
                    return false;
                tc::tc_fence_after();
                int c0, c1;
                changed(v - 1u, c0, c1);
                mma_chunks(v, q, c0, 4);
                mma_chunks(v, c1 + (((q - c1) % 4) + 4) % 4, kx, 4);
            }
            tc::mma_commit(mma_bar(v));
            return true;
        };
        bool ok = true;
        // Tile 0 goes out before any noise (block 0's GEMM needs it at once); tile u + 1 after
        // the noise of block u, a block ahead of its GEMM.  Its slot was freed by block
        // u + 1 - kFRing, which needs no noise this warp has yet to produce.
        if (stager) ok = stage(0u);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        for (uint32_t it = 0; ok && it < ndec; ++it) {
            const uint32_t slot = it & 1u;
            if (it >= 2 && !f_wait_warp(&bars[kFBarNoiseFree + 2 * q + slot],
                                        ((it >> 1) + 1u) & 1u, abort_flag, status, 0))
                break;
            const uint32_t t = it / (uint32_t)nb;
            const int s0 = (int)(it % (uint32_t)nb) * K;
            float *tb = thbuf + slot * K * kFLanes;
#pragma unroll 4
            for (int g4 = 0; g4 < K / 4; ++g4) {
                const uint4 rw = philox4x32_10(
                    make_uint4((uint32_t)((s0 >> 2) + g4), t, chain, iter), key0, key1);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    // Spins past N' (block padding) get a threshold that keeps them at 0.
                    const bool real = s0 + 4 * g4 + e < nprime;
                    tb[(4 * g4 + e) * kFLanes + r] = real ? theta_of_word(word_of(rw, e)) : -1e30f;
                }
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&bars[kFBarNoise + 2 * q + slot]);
            // Block it's part first: with two tile slots, staging tile it + 1 waits for the end of
            // block it - 1, and the part should run during that block.
            if (lane == 0) ok = issue_ahead(it);
            if (stager && ok && it + 1u < total) ok = stage(it + 1u);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        }
        // The readout pass (no noise): its tiles, and this warp's parts of its GEMMs.
        for (uint32_t v = ndec; ok && v < total; ++v) {
            if (stager)   // tile v (when the sweeps are few it may not be out yet)
                while (ok && tiles_issued <= v) ok = stage(tiles_issued);
            if (lane == 0 && ok) ok = issue_ahead(v);
            if (stager)
                while (ok && tiles_issued < total && tiles_issued <= v + 1u) ok = stage(tiles_issued);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        }
        // Every MMA this warp issued completes before the outputs and the TMEM release (bounded,
        // not cut short by an abort).
        if (lane == 0) {
            tc::mma_commit(&bars[kFBarNDrain + q]);
            f_wait(&bars[kFBarNDrain + q], 0, nullptr, status, 0);
        }
        // The copies complete before shared memory is released.
        if (stager)
            for (uint32_t ts = 0; ts < kFRing && ts < tiles_issued; ++ts) {
                const uint32_t uses = (tiles_issued - ts + kFRing - 1u) / kFRing;
                f_wait(&bars[kFBarTile + ts], (uses - 1u) & 1u, nullptr, status, 0);
            }
        __syncwarp();
    } else {
        if (kSplit) asm volatile("setmaxnreg.inc.sync.aligned.u32 192;");
        const int r = threadIdx.x;
        const int chain = grp * kFLanes + r;
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
        const float4 *__restrict__ spinc = ip->spinc;
        const float *lam = a.lambda + (size_t)j * a.m_stride;

        // End of block v - 1 (v = 0: the start) for this warp: its arrival; the last warp issues
        // the chunks block v - 1 changed (v < 2: every chunk) and commits.
        auto arrive_and_issue = [&](uint32_t *counter, uint32_t v, int c0, int c1) -> bool {
            bool ok2 = true;
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                const bool last = (atomicAdd(counter, 1u) & 3u) == 3u;
                if (last && v < total) {
                    __threadfence_block();
                    tc::tc_fence_after();
                    if (v < 2u) {   // no part was issued ahead: the whole GEMM
                        c0 = 0;
                        c1 = kx;
                    }
                    if (c1 > c0) {
                        ok2 = tile_ready(v);
                        if (ok2) mma_chunks(v, c0, c1, 1);
                    }
                    if (ok2) tc::mma_commit(mma_bar(v));
                }
            }
            return __shfl_sync(0xffffffffu, ok2 ? 1 : 0, 0) != 0;
        };
        // This warp's rows of an accumulator slot set to 0 (warp-collective).
        // Stores issued; the caller waits (tmem_wait_st) before its tile-free arrival.
        auto zero_slot = [&](uint32_t slot) {
#pragma unroll
            for (int c16 = 0; c16 < KD; c16 += 16)
                tc::tmem_zero16_nowait(lane_addr + dcol0 + slot * (uint32_t)KD + (uint32_t)c16);
        };

        // Every run starts from x = 0 (Sec. III-B): X and the bit-packed states cleared.
        for (int w = 0; w < xwords; ++w) xs[w * kFLanes + r] = 0u;
        {
            const uint32_t zero8[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            for (int c0 = 0; c0 < 8 * kxt; c0 += 8) tc::tmem_st8(lane_addr + (uint32_t)c0, zero8);
            for (int c = kxt; c < kx; ++c) {
                unsigned char *row = xsm + (size_t)(c - kxt) * kFXChunkBytes + (r >> 3) * 256 +
                                     (r & 7) * 16;
                *reinterpret_cast<uint4 *>(row) = make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4 *>(row + 128) = make_uint4(0u, 0u, 0u, 0u);
            }
            if (kx > kxt) tc::fence_proxy_async_smem();
            zero_slot(0u);
            zero_slot(1u);
            tc::tmem_wait_st();
        }
        bool ok = arrive_and_issue(&arrivals[2], 0u, 0, kx);

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
        // The constraint values as FP32 too (exact: |g| < 2^24, checked at creation), so that
        // the decision chain updates them and c_k without integer <-> float conversions.
        float gf[MC];
#pragma unroll
        for (int k = 0; k < MC; ++k) gf[k] = (float)g[k];
        const float errk = field_err_factor(m);
        // Fault-injection test (dec_wait_polls > 0): wait on a barrier nothing completes, so the
        // bound expires and the kernel takes its timeout path.
        if (ok && dec_wait_polls > 0)
            ok = f_wait_warp(&bars[kFBarNever], 0, abort_flag, status, dec_wait_polls);
        long long ccur = 0, rbest = LLONG_MAX;   // cost of the current state (kTrack)
        int rsweep = -1, rnf = 0;
        long long sumF = 0, sumh = 0;            // readout pass
        float Fr[K];
        for (uint32_t it = 0; ok && it < total; ++it) {
            const bool readout = it >= ndec;
            const uint32_t t = readout ? (uint32_t)a.sweeps : it / (uint32_t)nb;
            const int b = (int)(readout ? it - ndec : it % (uint32_t)nb);
            const int s0 = b * K;
            const uint32_t ts = f_slot(it, kFRing);
            const uint32_t slot = it & 1u;
            const float *thb = thbuf + slot * K * kFLanes + r;
            // the block's records and h: staged in shared memory (K >= 32) or global
            const float4 *scs =
                kSide ? reinterpret_cast<const float4 *>(ring + ts * slot_stride + side_off)
                      : spinc + s0;
            const float *hs = kSide ? reinterpret_cast<const float *>(ring + ts * slot_stride +
                                                                      side_off + (uint32_t)(K * 16))
                                    : hF + s0;
            // K = 16: the block's per-spin data, loaded before the wait for the block's GEMM,
            // which they overlap: the noise theta and the record {a_0i, D_i, sum_k a_ki, a_1i}.
            // Larger blocks load them spin by spin (registers).
            constexpr int kPre = K == 16 ? 16 : 1;
            float th16[kPre];
            float4 sc16[kPre];
            if (!readout) {
                // Noise of the block (partner noise warp) and its W tile (diagonal for the
                // in-block corrections).
                if (!f_wait_warp(&bars[kFBarNoise + 2 * warp + slot], (it >> 1) & 1u, abort_flag,
                                 status, dec_wait_polls) ||
                    !f_wait_warp(&bars[kFBarTile + ts], f_round(it, kFRing) & 1u, abort_flag, status,
                                 dec_wait_polls)) {
                    ok = false;
                    break;
                }
                if (K == 16) {   // the noise is in registers: its slot may be refilled
#pragma unroll
                    for (int ii = 0; ii < kPre; ++ii) {
                        th16[ii] = thb[ii * kFLanes];
                        sc16[ii] = scs[ii];
                    }
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&bars[kFBarNoiseFree + 2 * warp + slot]);
                }
            } else if (!f_wait_warp(&bars[kFBarTile + ts], f_round(it, kFRing) & 1u, abort_flag,
                                    status, dec_wait_polls)) {   // h of the block
                ok = false;
                break;
            }
            // This block's fields: its GEMM is done (issued by the last warp of the block before).
            if (!f_wait_warp(mma_bar(it), (it >> 1) & 1u, abort_flag, status, dec_wait_polls)) {
                ok = false;
                break;
            }
            tc::tc_fence_after();
            const uint32_t dcol = dcol0 + (it & 1u) * (uint32_t)KD;   // this block's slot
            f_load_fields<K, kHiLo>(lane_addr + dcol, Fr);
#pragma unroll
            for (int ii = 0; ii < K; ++ii) Fr[ii] += hs[ii];   // exact integers
            const int wi = s0 >> 5, sb = s0 & 31;
            if (readout) {
                // Readout pass: sum_i x_i F_i and h^T x over the block, from the final states.
                int32_t pf = 0, ph = 0;   // |F|, |h| < 2^24 and K <= 64 terms: exact in int32
#pragma unroll
                for (int ii = 0; ii < K; ++ii) {
                    const uint32_t xw = xs[((s0 + ii) >> 5) * kFLanes + r];
                    if ((xw >> ((s0 + ii) & 31)) & 1u) {
                        pf += __float2int_rz(Fr[ii]);
                        ph += __float2int_rz(hs[ii]);
                    }
                }
                sumF += pf;
                sumh += ph;
                zero_slot(it & 1u);   // for the GEMM of block it + 2
                tc::tmem_wait_st();
                tc::tc_fence_before();   // the noise warps' MMAs of block it + 2 follow
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&bars[kFBarTileFree + ts]);
                ok = arrive_and_issue(&arrivals[it & 1u], it + 1u, 0, 0);
                continue;
            }
            const float beta = beta_of_sweep(a.beta_max, (int)t, a.sweeps);
            const float hb = 0.5f * beta;
            const float ez = hb * errk;
            const float *wdg = reinterpret_cast<const float *>(ring + ts * slot_stride + diag_off);
            uint32_t xwv[kXW];
#pragma unroll
            for (int q = 0; q < kXW; ++q) xwv[q] = xs[(wi + q) * kFLanes + r];
            uint32_t xold[kXW];
#pragma unroll
            for (int q = 0; q < kXW; ++q) xold[q] = xwv[q];
            // Block-start chain state, kept for an exact re-run of the block.
            float gf0[MC], cb[MC];
            const float M0 = Mmax;
#pragma unroll
            for (int k = 0; k < MC; ++k) {
                gf0[k] = gf[k];
                cb[k] = c[k];
            }
            int32_t cblk = 0;   // cost change over the block (kTrack): |sum| < K 2^24 <= 2^30
            bool near_tie = false;
#pragma unroll
            for (int ii = 0; ii < K; ++ii) {
                const int s = s0 + ii;
                // word and bit of spin s in the block's state words (K = 16: one word, bit sb + ii;
                // K >= 32: blocks start on a word, so the word index is a constant)
                const int bw = K == 16 ? 0 : (ii >> 5), bi = K == 16 ? sb + ii : (ii & 31);
                const float4 sc = K == 16 ? sc16[ii % kPre] : scs[ii];
                // Row ii of the block's diagonal of W (FP32, the same address for every lane):
                // the quads right of spin ii, for the in-block corrections.
                float4 wq[K / 4];
#pragma unroll
                for (int q4 = (ii + 1) >> 2; q4 < K / 4; ++q4)
                    wq[q4] = *reinterpret_cast<const float4 *>(wdg + ii * K + 4 * q4);
                const float Fi = Fr[ii];
                const int xi = (xold[bw] >> bi) & 1;
                float akf[MC];
                float acc = sf * Fi;
                const float tabs = fabsf(acc);
#pragma unroll
                for (int k = 0; k < MC; ++k) {
                    if (k == 0)
                        akf[k] = sc.x;
                    else if (k == 1)
                        akf[k] = sc.w;
                    else
                        akf[k] = (k < m) ? (float)__ldg(acol + (size_t)s * m + k) : 0.f;
                    acc = fmaf(-akf[k], c[k], acc);
                }
                const float Di = sc.y;
                acc = fmaf(xi ? 1.f : -1.f, Di, acc);
                const float z = hb * acc;
                const float theta = K == 16 ? th16[ii % kPre] : thb[ii * kFLanes];
                const float y = z + theta;
                const float bound =
                    ez * (tabs + sc.z * Mmax + Di) + kThetaRelErr * fabsf(theta) + kThetaAbsErr;
                // A decision the FP32 bound cannot settle is only flagged here; the warp then
                // re-runs the block below with the FP64 path.
                near_tie |= !(fabsf(y) > bound);
                // The flip d = x_new - x_i in {-1, 0, +1}, kept as FP32.
                const float df = (y > 0.f ? 1.f : 0.f) - (xi ? 1.f : 0.f);
                if (kTrack) cblk -= __float2int_rz(df * Fi);
                xwv[bw] ^= (uint32_t)(df != 0.f) << bi;
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
                    // In-block correction F_jj += W[s, s0+jj] d for the block's later spins.  The
                    // next spin's field is on the dependency chain: corrected unconditionally (d =
                    // 0 adds an exact zero); the others only when a chain of the warp flipped.
                    auto wcol = [&](int jj) -> float {
                        const float4 &v = wq[jj >> 2];
                        const int e = jj & 3;
                        return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
                    };
                    Fr[ii + 1] = fmaf(df, wcol(ii + 1), Fr[ii + 1]);
                    if (ii + 2 < K && __any_sync(0xffffffffu, df != 0.f)) {
#pragma unroll
                        for (int jj = ii + 2; jj < K; ++jj) Fr[jj] = fmaf(df, wcol(jj), Fr[jj]);
                    }
                }
            }
            if (__any_sync(0xffffffffu, near_tie)) {
                // Exact re-run of the block for the whole warp, from its start state: the fields
                // from D (this block's GEMM result, unchanged until the next GEMM) plus h and the
                // block's earlier flips, the noise recomputed, the same FP32 evaluation, and FP64
                // where the bound cannot settle the decision.  Decisions outside near-ties come
                // out as before.
                // The block's bits as one word (bit ii = spin s0 + ii): start state and re-run state.
                uint64_t bo;
                if constexpr (K == 16)
                    bo = (xold[0] >> sb) & 0xFFFFu;
                else if constexpr (K == 32)
                    bo = xold[0];
                else
                    bo = (uint64_t)xold[0] | ((uint64_t)xold[kXW - 1] << 32);
                uint64_t bn = bo;
                Mmax = M0;
                cblk = 0;
#pragma unroll
                for (int k = 0; k < MC; ++k) {
                    g[k] = (int32_t)gf0[k];
                    c[k] = cb[k];
                }
#pragma unroll 1
                for (int ii = 0; ii < K; ++ii) {
                    const int s = s0 + ii;
                    uint32_t fv, fl_lo = 0u;
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                                 : "=r"(fv)
                                 : "r"(lane_addr + dcol + (uint32_t)ii));
                    if (kHiLo)
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                                     : "=r"(fl_lo)
                                     : "r"(lane_addr + dcol + (uint32_t)(K + ii)));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    float Fi = __uint_as_float(fv) + hs[ii];
                    if (kHiLo) Fi += __uint_as_float(fl_lo);
                    uint64_t fl = (bn ^ bo) & ((1ull << ii) - 1ull);
                    while (fl) {
                        const int i2 = __ffsll((long long)fl) - 1;
                        fl &= fl - 1ull;
                        const int d2 = (int)((bn >> i2) & 1ull) - (int)((bo >> i2) & 1ull);
                        Fi = fmaf((float)d2, wdg[ii * K + i2], Fi);
                    }
                    const int xi = (int)((bo >> ii) & 1ull);
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
                        make_uint4((uint32_t)(s >> 2), t, (uint32_t)chain, iter), key0, key1);
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
                    if (kTrack) cblk -= d * __float2int_rz(Fi);
                    bn ^= (uint64_t)(d != 0) << ii;
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
                if constexpr (K == 16) {
                    xwv[0] = (xold[0] & ~(0xFFFFu << sb)) | ((uint32_t)bn << sb);
                } else {
                    xwv[0] = (uint32_t)bn;
                    if constexpr (kXW > 1) xwv[kXW - 1] = (uint32_t)(bn >> 32);
                }
            }
            if (kTrack) ccur += cblk;
#pragma unroll
            for (int q = 0; q < kXW; ++q) xs[(wi + q) * kFLanes + r] = xwv[q];
            // The block's new states into X (item spins only; BF16 1.0 = 0x3F80), for the GEMMs of
            // the blocks after it.
            if (s0 < n16) {
#pragma unroll
                for (int h8 = 0; h8 < K / 16; ++h8) {
                    if (s0 + 16 * h8 < n16) {
                        uint32_t v8[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int i0 = 16 * h8 + 2 * e;   // spin s0 + i0 and the next one
                            const uint32_t w0 = xwv[K == 16 ? 0 : (i0 >> 5)];
                            const int sh = K == 16 ? sb + i0 : (i0 & 31);
                            v8[e] = (((w0 >> sh) & 1u) ? 0x3F80u : 0u) |
                                    (((w0 >> (sh + 1)) & 1u) ? 0x3F800000u : 0u);
                        }
                        const int c = (s0 >> 4) + h8;   // the 16-spin chunk
                        if (c < kxt) {
                            tc::tmem_st8_nowait(lane_addr + (uint32_t)(8 * c), v8);
                        } else {
                            unsigned char *row = xsm + (size_t)(c - kxt) * kFXChunkBytes +
                                                 (r >> 3) * 256 + (r & 7) * 16;
                            *reinterpret_cast<uint4 *>(row) = make_uint4(v8[0], v8[1], v8[2], v8[3]);
                            *reinterpret_cast<uint4 *>(row + 128) =
                                make_uint4(v8[4], v8[5], v8[6], v8[7]);
                            tc::fence_proxy_async_smem();   // for the next block's MMAs
                        }
                    }
                }
            }
            zero_slot(it & 1u);   // for the GEMM of block it + 2
            tc::tmem_wait_st();      // the state chunk and the zeros
            tc::tc_fence_before();   // the noise warps' MMAs of block it + 2 follow
            __syncwarp();
            if (lane == 0) {
                if (K != 16) tc::mbar_arrive(&bars[kFBarNoiseFree + 2 * warp + slot]);
                tc::mbar_arrive(&bars[kFBarTileFree + ts]);
            }
            {
                int c0, c1;
                changed(it, c0, c1);
                ok = arrive_and_issue(&arrivals[it & 1u], it + 1u, c0, c1);
            }
            // Sweep end: best feasible sweep-end state of the run, and the trace.
            if (ok && b == nb - 1) {
                if (kTrack) {
                    bool feas = true;
#pragma unroll
                    for (int k = 0; k < MC; ++k) {
                        if (k < m) {
                            const int o0 = ip->slack_off[k], o1 = ip->slack_off[k + 1];
                            long long sv = 0;
                            for (int s = o0; s < o1; ++s)
                                if ((xs[(s >> 5) * kFLanes + r] >> (s & 31)) & 1u)
                                    sv += 1LL << (s - o0);
                            if ((long long)gf[k] - sv > (long long)ip->fmargin[k]) feas = false;
                        }
                    }
                    if (feas) {
                        ++rnf;
                        if (ccur < rbest) {
                            rbest = ccur;
                            rsweep = (int)t;
                            if (valid) {
                                uint32_t *rx = a.run_x + ((size_t)j * a.chains + chain) * a.words;
                                for (int w = 0; w < a.words; ++w)
                                    rx[w] = w < words ? xs[w * kFLanes + r] : 0u;
                            }
                        }
                    }
                }
                if (a.trace && valid) {
                    uint32_t *tr =
                        a.trace + (((size_t)j * a.chains + chain) * a.sweeps + t) * a.words;
                    for (int w = 0; w < a.words; ++w) tr[w] = w < words ? xs[w * kFLanes + r] : 0u;
                }
            }
        }
        // Drain: every MMA of the CTA completes before the outputs and the TMEM release.  Each
        // decision warp's lane 0 commits the MMAs it issued; every warp waits for all four,
        // bounded but not cut short by an abort.
        if (lane == 0) tc::mma_commit(&bars[kFBarDrain + warp]);
        __syncwarp();
        bool drained = true;
        if (lane == 0)
            for (int w = 0; w < 4; ++w)
                drained = f_wait(&bars[kFBarDrain + w], 0, nullptr, status, 0) && drained;
        drained = __shfl_sync(0xffffffffu, drained ? 1 : 0, 0) != 0;
        tc::tc_fence_after();
        if (ok && drained && valid) {
#pragma unroll
            for (int k = 0; k < MC; ++k) g[k] = (int32_t)gf[k];
            const size_t cidx = (size_t)j * a.chains + chain;
            for (int w = 0; w < a.words; ++w)
                a.x[cidx * a.words + w] = w < words ? xs[w * kFLanes + r] : 0u;
            a.cost[cidx] = -(sumF + sumh) / 2;
            bool feas = true;
#pragma unroll
            for (int k = 0; k < MC; ++k) {
                if (k < m) {
                    const int o0 = ip->slack_off[k], o1 = ip->slack_off[k + 1];
                    long long sv = 0;
                    for (int s = o0; s < o1; ++s)
                        if ((xs[(s >> 5) * kFLanes + r] >> (s & 31)) & 1u) sv += 1LL << (s - o0);
                    if ((long long)g[k] - sv > (long long)ip->fmargin[k]) feas = false;
                    a.g[cidx * a.m_stride + k] = g[k];
                }
            }
            for (int k = m; k < a.m_stride; ++k) a.g[cidx * a.m_stride + k] = 0;
            if (a.feasible) a.feasible[cidx] = feas ? 1 : 0;
            if (kTrack) {
                a.run_cost[cidx] = rbest;
                if (a.run_sweep) a.run_sweep[cidx] = rsweep;
                if (a.run_nfeas) a.run_nfeas[cidx] = rnf;
                if (rsweep < 0)
                    for (int w = 0; w < a.words; ++w) a.run_x[cidx * a.words + w] = 0u;
            }
        }
    }
    // Every TMEM access and copy of the item is over before the next item or the release.
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const bool done = *abort_flag == 0;
    // A completed item's barriers have no operation pending: end them, so that the next item
    // may initialise barriers or keep plain data there.  (After an abort the CTA stops.)
    if (done && threadIdx.x == 0)
        for (int i = 0; i < kFBars; ++i) tc::mbar_inval(&bars[i]);
    return done;
}

// One launch of the block-field sampler: one work item per CTA (the work list's (instance,
// chain group), or the grid's), TMEM held for the CTA's life.
template <int MC, int K, bool kHiLo, bool kTrack>
__global__ void __launch_bounds__(kFThreads, 2)
    field_sampler_kernel(SampleArgs a, int32_t *status, long long dec_wait_polls, FieldLaunch L) {
    extern __shared__ __align__(1024) unsigned char smem[];
    // The TMEM address is written to the first word of shared memory and read by every thread
    // before the item starts to use that memory.
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem);
    const int j = a.work ? a.work[2 * blockIdx.x] : (int)blockIdx.y;
    const int grp = a.work ? a.work[2 * blockIdx.x + 1] : (int)blockIdx.x;
    if (threadIdx.x < 32) {
        tc::tmem_alloc(tmem_slot, L.cols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    __syncthreads();
    field_item<MC, K, kHiLo, kTrack, true>(a, j, grp, tmem, L, status, dec_wait_polls);
    if (threadIdx.x < 32) tc::tmem_dealloc(tmem, L.cols);
}

template <int MC, int K, bool H, bool T>
cudaError_t field_launch(const SampleArgs &a, int32_t *status, long long polls,
                         const FieldLaunch &L, cudaStream_t s) {
    auto kern = field_sampler_kernel<MC, K, H, T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L.smem);
    if (e != cudaSuccess) return e;
    const dim3 grid = a.work ? dim3(a.nwork, 1) : dim3((a.chains + kFLanes - 1) / kFLanes, a.count);
    kern<<<grid, kFThreads, L.smem, s>>>(a, status, polls, L);
    return cudaGetLastError();
}

template <int K, bool H, bool T>
cudaError_t field_launch_mc(const SampleArgs &a, int max_m, int32_t *status, long long polls,
                            const FieldLaunch &L, cudaStream_t s) {
    if (max_m <= 1) return field_launch<1, K, H, T>(a, status, polls, L, s);
    if (max_m <= 2) return field_launch<2, K, H, T>(a, status, polls, L, s);
    if (max_m <= 4) return field_launch<4, K, H, T>(a, status, polls, L, s);
    return field_launch<8, K, H, T>(a, status, polls, L, s);   // m <= 8
}

}  // namespace
}  // namespace sais
