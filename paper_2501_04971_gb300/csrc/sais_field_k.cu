// sais_field_k.cu -- the block-field p-bit sampler with K = 32 and K = 64 spins per block, for
// instances with at most two constraints (kernel in sais_field_kernel.cuh, launch in
// sais_field.cu).
#include "sais_field_kernel.cuh"

namespace sais {

namespace {
template <int K>
cudaError_t wide_k(const SampleArgs &a, int max_m, bool hilo, bool track, int32_t *status,
                   long long polls, const FieldLaunch &L, cudaStream_t st) {
    if (max_m <= 1) {
        if (hilo)
            return track ? field_launch<1, K, true, true>(a, status, polls, L, st)
                         : field_launch<1, K, true, false>(a, status, polls, L, st);
        return track ? field_launch<1, K, false, true>(a, status, polls, L, st)
                     : field_launch<1, K, false, false>(a, status, polls, L, st);
    }
    if (hilo)
        return track ? field_launch<2, K, true, true>(a, status, polls, L, st)
                     : field_launch<2, K, true, false>(a, status, polls, L, st);
    return track ? field_launch<2, K, false, true>(a, status, polls, L, st)
                 : field_launch<2, K, false, false>(a, status, polls, L, st);
}
}  // namespace

cudaError_t launch_field_wide(const SampleArgs &a, int max_m, int block_k, bool hilo, bool track,
                              int32_t *status, long long polls, const FieldLaunch &L,
                              cudaStream_t st) {
    if (max_m > 2) return cudaErrorInvalidValue;   // the host admits m <= 2 for K = 32, 64
    if (block_k == 32)
        return wide_k<32>(a, max_m, hilo, track, status, polls, L, st);
    return wide_k<64>(a, max_m, hilo, track, status, polls, L, st);
}

}  // namespace sais
