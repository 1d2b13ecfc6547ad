// sais_ragged.cu -- launch of the persistent ragged-batch kernel (sais_ragged_kernel.cuh), the
// variant without the BF16 hi/lo split; sais_ragged_hilo.cu holds the other.
#include "sais_ragged_kernel.cuh"

namespace sais {

cudaError_t launch_ragged_hilo(const SampleArgs &a, const int32_t *items, int32_t nitems,
                               int32_t *head, unsigned long long *stats, const FieldLaunch &L,
                               int grid, int32_t *status, long long polls, cudaStream_t st);

size_t ragged_smem_bytes(int max_n16_w, int max_words, bool hilo, int *ring) {
    size_t f = 0;
    *ring = 3;
    if (max_n16_w > 0) {
        *ring = field_ring(max_n16_w, max_words, 16, hilo);
        f = field_smem_bytes(max_n16_w, max_words, 16, hilo);
    }
    const size_t p = plain_smem_bytes(0, max_words, false, kRaggedPlainChains);
    return std::max(f, p);
}

int ragged_grid(int nitems, int sms) { return std::max(1, std::min(nitems, sms)); }

cudaError_t launch_ragged(const SampleArgs &a, const int32_t *items, int32_t nitems,
                          int32_t *head, unsigned long long *stats, int max_n16_w,
                          int max_words, bool hilo, int32_t *status, long long dec_wait_polls,
                          int sms, cudaStream_t st) {
    FieldLaunch L;
    L.cols = 512;
    L.max_n16 = std::max(16, max_n16_w);
    L.xs_chunks = max_n16_w > 0 ? field_xs_chunks(max_n16_w, field_dcols(16, hilo)) : 0;
    int ring = 3;
    L.smem = ragged_smem_bytes(max_n16_w, max_words, hilo, &ring);
    L.ring = ring;
    // one CTA per SM: the shared-memory request leaves no room for a second
    const size_t floor_smem = (size_t)228 * 1024 / 2 + 1;
    if (L.smem < floor_smem) L.smem = floor_smem;
    const long long polls = dec_wait_polls > 0 ? dec_wait_polls : 0;
    const int grid = ragged_grid(nitems, sms);
    if (hilo) return launch_ragged_hilo(a, items, nitems, head, stats, L, grid, status, polls, st);
    return ragged_launch_h<false>(a, items, nitems, head, stats, L, grid, status, polls, st);
}

}  // namespace sais
