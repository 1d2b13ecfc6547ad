// sais_blocked_stream.cu -- the blocked p-bit sampler variants that stream W tiles through a
// shared-memory ring (N'_pad beyond the resident limit, and the BF16 hi/lo split for pair
// values above 256).  Kernel in sais_blocked_kernel.cuh.
#include "sais_blocked_kernel.cuh"

namespace sais {

cudaError_t launch_blocked_stream(const SampleArgs &a, int max_m, bool hilo, int32_t *status,
                                  long long polls, size_t smem, uint32_t cols, cudaStream_t st) {
    if (!hilo) return launch_mc<16, true, false>(a, max_m, status, polls, smem, cols, st);
    return launch_mc<16, true, true>(a, max_m, status, polls, smem, cols, st);
}

}  // namespace sais
