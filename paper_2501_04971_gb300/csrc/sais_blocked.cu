// sais_blocked.cu -- blocked p-bit sampler with the rank-k field update on the tensor cores.
#include "sais_device.cuh"

namespace sais {

cudaError_t launch_blocked_sampler(const SampleArgs &, int, int, int, int, cudaStream_t,
                                   const char **why_unsupported) {
    *why_unsupported = "the blocked sampler is not available in this build";
    return cudaSuccess;
}

}  // namespace sais
