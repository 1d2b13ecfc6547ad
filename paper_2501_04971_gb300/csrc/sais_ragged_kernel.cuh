// sais_ragged_kernel.cuh -- one persistent launch for a ragged batch (SAIS_AUTO).
//
// The batch's work is a list of items, (instance, chain group, kind), sorted most expensive
// first on the host.  The launch has one CTA of 256 threads per SM (TMEM: 512 columns held for
// the CTA's life); each CTA takes the next item from a device counter (one atomicAdd, no wait)
// and runs it to the end, so an SM that finishes early takes more work instead of idling:
//   kind 0 / 1  quadratic objective, m <= 1 / m <= 8: the block-field sampler on 128 chains
//               (field_item, K = 16): the fields of each block from one tcgen05 GEMM over the
//               states, in-block corrections on CUDA cores;
//   kind 2 / 3  linear objective, m <= 8 / m <= 32: the plain sampler on 256 chains, one per
//               thread (plain_item).
// Every chain is the sequential Gibbs sweep of Sec. III-B whichever kernel runs it, so the results
// equal those of the per-group launches element by element.  A bounded wait that gives up inside
// an item records SAIS_ETIMEOUT; that CTA then takes no further item.  Each CTA records, on the
// GPU's global timer, when it started and ended, the time it spent inside items and how many it
// ran (4 x uint64 per CTA), so the host can see how evenly the SMs were kept busy.
#pragma once

#include "sais_field_kernel.cuh"
#include "sais_plain_item.cuh"

namespace sais {
namespace {

constexpr int kRaggedThreads = 256;
constexpr int kRaggedPlainChains = 256;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <bool kHiLo, bool kTrack>
__global__ void __launch_bounds__(kRaggedThreads, 1)
    ragged_kernel(SampleArgs a, const int32_t *items, int32_t nitems, int32_t *head,
                  unsigned long long *stats, FieldLaunch L, int32_t *status,
                  long long dec_wait_polls) {
    extern __shared__ __align__(1024) unsigned char smem[];
    // The TMEM address and each item's index pass through the first two words of shared
    // memory; every thread reads them before an item uses that memory.
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem);
    volatile int32_t *item_s = reinterpret_cast<volatile int32_t *>(smem + 4);
    const unsigned long long t_start = global_ns();
    unsigned long long busy = 0, t_item = 0, n_items = 0;
    if (threadIdx.x < 32) {
        tc::tmem_alloc(tmem_slot, L.cols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long now = global_ns();
            if (n_items) busy += now - t_item;
            t_item = now;
            *item_s = atomicAdd(head, 1);
        }
        __syncthreads();
        const int32_t it = *item_s;
        __syncthreads();   // every thread has read the index before thread 0 takes the next
        if (it >= nitems) break;
        ++n_items;
        const int j = items[3 * it], grp = items[3 * it + 1], kind = items[3 * it + 2];
        if (!SAIS_DCHECK(status, it >= 0 && kind >= 0 && kind <= 3)) break;
        bool ok = true;
        if (kind == 0)
            ok = field_item<1, 16, kHiLo, kTrack, false>(a, j, grp, tmem, L, status,
                                                         dec_wait_polls);
        else if (kind == 1)
            ok = field_item<8, 16, kHiLo, kTrack, false>(a, j, grp, tmem, L, status,
                                                         dec_wait_polls);
        else if (kind == 2)
            plain_item<8>(a, j, grp, kRaggedPlainChains, (int)threadIdx.x);
        else
            plain_item<32>(a, j, grp, kRaggedPlainChains, (int)threadIdx.x);
        __syncthreads();
        if (!ok) {
            if (threadIdx.x == 0) busy += global_ns() - t_item;
            break;
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, L.cols);
    }
    if (threadIdx.x == 0) {
        unsigned long long *s = stats + 4 * blockIdx.x;
        s[0] = t_start;
        s[1] = global_ns();
        s[2] = busy;
        s[3] = n_items;
    }
}

template <bool H>
cudaError_t ragged_launch_h(const SampleArgs &a, const int32_t *items, int32_t nitems,
                            int32_t *head, unsigned long long *stats, const FieldLaunch &L,
                            int grid, int32_t *status, long long polls, cudaStream_t st) {
    const bool track = a.run_cost != nullptr;
    auto kern = track ? ragged_kernel<H, true> : ragged_kernel<H, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L.smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(head, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    kern<<<grid, kRaggedThreads, L.smem, st>>>(a, items, nitems, head, stats, L, status, polls);
    return cudaGetLastError();
}

}  // namespace
}  // namespace sais
