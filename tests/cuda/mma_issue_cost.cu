// mma_issue_cost.cu -- cost of tcgen05.mma instructions as the block-field and rank-k samplers
// issue them (a measurement, not a correctness check).
//
// One CTA per SM (152 at once) issues R MMAs of M = 128, K = 16, BF16 with FP32 accumulation
// from one thread, commits them to an mbarrier and waits; clock64 from the first issue to the
// commit's completion, mean of `reps` repetitions after two untimed ones.  Two series:
//   chain  R accumulating MMAs into one accumulator, N in {16, 32, 64, 128, 256}, A from TMEM
//          or from shared memory;
//   split  19 MMAs (N = 16, 32) spread round-robin over P independent accumulators.
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
__global__ void __launch_bounds__(128, 1) probe(long long *out, int N, int R, int a_smem, int P,
                                                int mode, int reps) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *B = smem;                  // N x 16 BF16, K-major: N * 32 bytes (N <= 256)
    unsigned char *A = smem + 256 * 32;       // 128 x 16 BF16: 4096 bytes
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 256 * 32 + 128 * 32);
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 1);
    for (int i = threadIdx.x; i < (256 * 32 + 128 * 32) / 4; i += blockDim.x)
        reinterpret_cast<uint32_t *>(smem)[i] = 0;
    if (threadIdx.x == 0) {
        tc::mbar_init(bar, 1);
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
    if (threadIdx.x == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(128, (uint32_t)N);
        const uint64_t bd = tc::smem_desc(tc::smem_u32(B), (uint32_t)N * 16u, 128u);
        const uint64_t ad = tc::smem_desc(tc::smem_u32(A), 128u * 16u, 128u);
        long long total = 0;
        bool ok = true;
        for (int rep = 0; rep < reps + 2 && ok; ++rep) {
            const long long t0 = clock64();
            for (int r = 0; r < R; ++r) {
                // A columns 8 (r % 19) + 0..7 < 160; accumulators from column 160 (mode 1) or
                // 256 (mode 0): 160 + 19 * 16 <= 512 and 256 + 256 <= 512
                if (mode == 1)
                    tc::mma_bf16_tmem_a(tmem + 160u + (uint32_t)((r % P) * N),
                                        tmem + 8u * (uint32_t)(r % 19), bd, idesc, r >= P);
                else if (a_smem)
                    tc::mma_bf16(tmem + 256u, ad, bd, idesc, r > 0);
                else
                    tc::mma_bf16_tmem_a(tmem + 256u, tmem + 8u * (uint32_t)(r % 19), bd, idesc,
                                        r > 0);
            }
            tc::mma_commit(bar);
            ok = wait_commit(bar, rep & 1);
            const long long t1 = clock64();
            if (rep >= 2) total += t1 - t0;
        }
        out[blockIdx.x] = ok ? total / reps : -1;
    }
    tc::tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

long long run(long long *d, int N, int R, int a_smem, int P, int mode) {
    static long long h[152];
    probe<<<152, 128, 200 * 1024>>>(d, N, R, a_smem, P, mode, 20);
    if (cudaDeviceSynchronize() != cudaSuccess) return -2;
    cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
    long long sum = 0;
    for (int i = 0; i < 152; ++i) {
        if (h[i] < 0) return -1;
        sum += h[i];
    }
    return sum / 152;
}

}  // namespace

int main() {
    long long *d = nullptr;
    if (cudaMalloc(&d, 152 * sizeof(long long)) != cudaSuccess) return 1;
    cudaFuncSetAttribute(probe, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    int bad = 0;
    for (int a_smem = 0; a_smem < 2; ++a_smem)
        for (int N : {16, 32, 64, 128, 256})
            for (int R : {1, 4, 19, 38}) {
                const long long c = run(d, N, R, a_smem, 1, 0);
                bad += c < 0;
                printf("chain A=%s N=%d R=%d cycles=%lld\n", a_smem ? "smem" : "tmem", N, R, c);
            }
    for (int N : {16, 32})
        for (int P : {1, 2, 4, 8, 19}) {
            if (160 + P * N > 512) continue;
            const long long c = run(d, N, 19, 0, P, 1);
            bad += c < 0;
            printf("split N=%d R=19 P=%d cycles=%lld\n", N, P, c);
        }
    cudaFree(d);
    return bad ? 2 : 0;
}
