// sais_blocked.cu -- launch of the blocked p-bit sampler (kernel in sais_blocked_kernel.cuh):
// shared-memory size, TMEM columns, and the variants with W resident in shared memory.  The
// variants that stream W tiles are instantiated in sais_blocked_stream.cu.
#include "sais_blocked_kernel.cuh"

namespace sais {

cudaError_t launch_blocked_stream(const SampleArgs &a, int max_m, bool hilo, int32_t *status,
                                  long long polls, size_t smem, uint32_t cols, cudaStream_t st);

size_t blocked_smem_bytes(int max_npad, int max_words, int block_k, bool stream, bool hilo) {
    const size_t w = stream ? (size_t)3 * (hilo ? 2 : 1) * (block_k / 8) * max_npad * 16
                            : (size_t)max_npad * max_npad * 2;
    return w + (size_t)max_words * kLanes * 4 + (size_t)2 * block_k * kLanes * 4 + 30 * 8 + 32;
}

cudaError_t launch_blocked_sampler(const SampleArgs &a, int max_m, int max_npad, int max_words,
                                   int block_k, bool stream, bool hilo, int32_t *status,
                                   long long dec_wait_polls, cudaStream_t st) {
    // TMEM columns: the power of two >= N'_pad + K (F, then the A operand).  At most 512 / cols
    // CTAs may share an SM, or a CTA's allocation would wait for another CTA's release; the
    // shared-memory request is raised so that no more CTAs than that fit on one SM.
    uint32_t cols = 32;
    while (cols < (uint32_t)(max_npad + block_k)) cols <<= 1;
    const size_t per_sm = 228 * 1024, max_ctas = 512 / cols;
    size_t smem = blocked_smem_bytes(max_npad, max_words, block_k, stream, hilo);
    const size_t floor_smem = per_sm / (max_ctas + 1) + 1;
    if (smem < floor_smem) smem = floor_smem;
    const long long polls = dec_wait_polls > 0 ? dec_wait_polls : 0;
    if (block_k == 32) return launch_mc<32, false, false>(a, max_m, status, polls, smem, cols, st);
    if (!stream) return launch_mc<16, false, false>(a, max_m, status, polls, smem, cols, st);
    return launch_blocked_stream(a, max_m, hilo, status, polls, smem, cols, st);
}

}  // namespace sais
