// mma_issue_cost.cu -- cost of tcgen05.mma instructions as the block-field and rank-k samplers
// issue them (a measurement, not a correctness check).
//
// One CTA per SM (152 at once) issues R MMAs of M = 128, K = 16, BF16 with FP32 accumulation
// from one thread, commits them to an mbarrier and waits; clock64 from the first issue to the
// commit's completion, mean of `reps` repetitions after two untimed ones, and separately the
// cycles the issuing thread spends in its R issue instructions (it stalls once the tensor
// pipe's queue is full).  Two series:
//   chain  R accumulating MMAs into one accumulator, N in {16, 32, 64, 128, 256}, A from TMEM
//          or from shared memory;
//   split  19 MMAs (N = 16, 32) spread round-robin over P independent accumulators;
//   warps  R MMAs issued by each of W warps (lane 0 of each, at once), each warp into its own
//          accumulator and committing to its own mbarrier: does a second issuing warp add
//          tensor throughput?  (same: every warp into one accumulator.)
// Every wait is bounded; on expiry the CTA records -1, waits once more (bounded) and frees TMEM.
#include <cstdio>
#include <cstdint>
#include "sais_tc.cuh"
using namespace sais;

namespace {

constexpr long long kPollLimit = 100000000ll;

__device__ bool wait_commit(uint64_t *bar, uint32_t parity) {
    long long polls = 0;
    while (!tc::mbar_try_wait(bar, parity) && ++polls < kPollLimit) {}
    if (polls < kPollLimit) return true;
    for (long long q = 0; q < kPollLimit && !tc::mbar_try_wait(bar, parity); ++q) {}
    return false;
}

// mode 0: R MMAs accumulating into one region (A from TMEM, or from shared memory if a_smem);
// mode 1: R MMAs round-robin over P regions (A from TMEM).
__global__ void __launch_bounds__(128, 1) probe(long long *out, long long *issue, int N, int R,
                                                int a_smem, int P, int mode, int reps) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *B = smem;                  // N x 16 BF16, K-major: N * 32 bytes (N <= 256)
    unsigned char *A = smem + 256 * 32;       // 128 x 16 BF16: 4096 bytes
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 256 * 32 + 128 * 32);   // [4]
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 4);
    for (int i = threadIdx.x; i < (256 * 32 + 128 * 32) / 4; i += blockDim.x)
        reinterpret_cast<uint32_t *>(smem)[i] = 0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < 4; ++w) tc::mbar_init(&bar[w], 1);
        tc::fence_mbar_init();
        out[blockIdx.x] = 0;
    }
    tc::fence_proxy_async_smem();
    if (threadIdx.x < 32) {
        tc::tmem_alloc(slot, 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *slot;
    if (mode == 2 || mode == 3) {
        // P warps issue R MMAs each (N <= 64: accumulators at 256 + 64 w, or all at 256 in
        // mode 3); warp 0 times them.
        const int w = threadIdx.x >> 5;
        const uint32_t idesc = tc::idesc_bf16_f32(128, (uint32_t)N);
        const uint64_t bd = tc::smem_desc(tc::smem_u32(B), (uint32_t)N * 16u, 128u);
        long long total = 0, t0 = 0;
        bool ok = true;
        for (int rep = 0; rep < reps + 2; ++rep) {
            __syncthreads();
            if (threadIdx.x == 0) t0 = clock64();
            if (w < P && (threadIdx.x & 31) == 0) {
                for (int r = 0; r < R; ++r)
                    tc::mma_bf16_tmem_a(tmem + 256u + (mode == 2 ? 64u * (uint32_t)w : 0u),
                                        tmem + 8u * (uint32_t)(r % 19), bd, idesc, 1u);
                tc::mma_commit(&bar[w]);
                ok = wait_commit(&bar[w], rep & 1) && ok;
            }
            __syncthreads();
            if (threadIdx.x == 0 && rep >= 2) total += clock64() - t0;
        }
        ok = __syncthreads_and(ok ? 1 : 0) != 0;
        if (threadIdx.x == 0) {
            out[blockIdx.x] = ok ? total / reps : -1;
            issue[blockIdx.x] = 0;
        }
    } else if (threadIdx.x == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(128, (uint32_t)N);
        const uint64_t bd = tc::smem_desc(tc::smem_u32(B), (uint32_t)N * 16u, 128u);
        const uint64_t ad = tc::smem_desc(tc::smem_u32(A), 128u * 16u, 128u);
        long long total = 0, total_issue = 0;
        bool ok = true;
        for (int rep = 0; rep < reps + 2 && ok; ++rep) {
            const long long t0 = clock64();
            // A columns 8 (r % 19) + 0..7 < 160; accumulators from column 160 (mode 1) or 256
            // (mode 0): 160 + 19 * 16 <= 512 and 256 + 256 <= 512.  One loop per form: a branch
            // around the MMA inside the loop slows the issue by itself.
            if (mode == 1)
                for (int r = 0; r < R; ++r)
                    tc::mma_bf16_tmem_a(tmem + 160u + (uint32_t)((r % P) * N),
                                        tmem + 8u * (uint32_t)(r % 19), bd, idesc, r >= P);
            else if (a_smem)
                for (int r = 0; r < R; ++r) tc::mma_bf16(tmem + 256u, ad, bd, idesc, r > 0);
            else
                for (int r = 0; r < R; ++r)
                    tc::mma_bf16_tmem_a(tmem + 256u, tmem + 8u * (uint32_t)(r % 19), bd, idesc,
                                        r > 0);
            const long long ti = clock64();
            tc::mma_commit(bar);
            ok = wait_commit(bar, rep & 1);
            const long long t1 = clock64();
            if (rep >= 2) {
                total += t1 - t0;
                total_issue += ti - t0;
            }
        }
        out[blockIdx.x] = ok ? total / reps : -1;
        issue[blockIdx.x] = total_issue / reps;
    }
    tc::tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

long long run(long long *d, int N, int R, int a_smem, int P, int mode, long long *issue_mean) {
    static long long h[152], hi[152];
    probe<<<152, 128, 200 * 1024>>>(d, d + 152, N, R, a_smem, P, mode, 20);
    if (cudaDeviceSynchronize() != cudaSuccess) return -2;
    cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
    cudaMemcpy(hi, d + 152, sizeof hi, cudaMemcpyDeviceToHost);
    long long sum = 0, si = 0;
    for (int i = 0; i < 152; ++i) {
        if (h[i] < 0) return -1;
        sum += h[i];
        si += hi[i];
    }
    *issue_mean = si / 152;
    return sum / 152;
}

}  // namespace

int main() {
    long long *d = nullptr;
    if (cudaMalloc(&d, 2 * 152 * sizeof(long long)) != cudaSuccess) return 1;
    cudaFuncSetAttribute(probe, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    int bad = 0;
    for (int a_smem = 0; a_smem < 2; ++a_smem)
        for (int N : {16, 32, 64, 128, 256})
            for (int R : {1, 4, 8, 19, 38, 56}) {
                long long is = 0;
                const long long c = run(d, N, R, a_smem, 1, 0, &is);
                bad += c < 0;
                printf("chain A=%s N=%d R=%d cycles=%lld issue=%lld\n", a_smem ? "smem" : "tmem",
                       N, R, c, is);
            }
    for (int N : {16, 64})
        for (int P : {1, 2, 4})
            for (int R : {19, 56}) {
                long long is = 0;
                const long long c = run(d, N, R, 0, P, 2, &is);
                bad += c < 0;
                printf("warps N=%d R=%d W=%d cycles=%lld\n", N, R, P, c);
                const long long c3 = run(d, N, R, 0, P, 3, &is);
                bad += c3 < 0;
                printf("same N=%d R=%d W=%d cycles=%lld\n", N, R, P, c3);
            }
    for (int N : {16, 32})
        for (int P : {1, 2, 4, 8, 19}) {
            if (160 + P * N > 512) continue;
            long long is = 0;
            const long long c = run(d, N, 19, 0, P, 1, &is);
            bad += c < 0;
            printf("split N=%d R=19 P=%d cycles=%lld issue=%lld\n", N, P, c, is);
        }
    cudaFree(d);
    return bad ? 2 : 0;
}
