// sais_field.cu -- launch of the block-field p-bit sampler (kernel in sais_field_kernel.cuh):
// shared-memory size, TMEM columns, CTAs per SM, and the block size K = 16 instantiations.  The
// K = 32 and K = 64 instantiations are in sais_field_k.cu.
#include "sais_field_kernel.cuh"

namespace sais {

cudaError_t launch_field_wide(const SampleArgs &a, int max_m, int block_k, bool hilo, bool track,
                              int32_t *status, long long polls, const FieldLaunch &L,
                              cudaStream_t st);

// TMEM columns: the power of two >= the state columns (8 per 16 item spins) plus K fields, at
// most 512 (state chunks beyond them live in shared memory).
uint32_t field_tmem_cols(int max_n16, int dcols) {
    uint32_t cols = 32;
    while (cols < 512u && cols < (uint32_t)(max_n16 / 2 + dcols)) cols <<= 1;
    return cols;
}

// 16-spin state chunks that do not fit TMEM beside the dcols accumulator columns.
int field_xs_chunks(int max_n16, int dcols) {
    const int in_tmem = (int)(field_tmem_cols(max_n16, dcols) - (uint32_t)dcols) / 8;
    return std::max(0, max_n16 / 16 - in_tmem);
}

size_t field_smem_ring(int max_n16, int max_words, int block_k, bool hilo, int ring) {
    // a tile slot: the W tile(s), the FP32 diagonal block, and for K >= 32 the per-spin records
    // and h
    const size_t slot = (size_t)block_k * max_n16 * 2 * (hilo ? 2 : 1) +
                        (size_t)block_k * block_k * 4 + (block_k >= 32 ? (size_t)block_k * 20 : 0);
    const size_t xwords = (size_t)((max_words + 1) & ~1);   // as the kernel rounds them
    return ring * slot + (size_t)field_xs_chunks(max_n16, field_dcols(block_k, hilo)) * kFXChunkBytes +
           xwords * kFLanes * 4 + (size_t)2 * block_k * kFLanes * 4 + kFBars * 8 + 32;
}

// Three W tile slots when they fit (the stager may run two blocks ahead), else two.
int field_ring(int max_n16, int max_words, int block_k, bool hilo) {
    return field_smem_ring(max_n16, max_words, block_k, hilo, 3) <= kMaxSmemPerBlock ? 3 : 2;
}

size_t field_smem_bytes(int max_n16, int max_words, int block_k, bool hilo) {
    return field_smem_ring(max_n16, max_words, block_k, hilo,
                           field_ring(max_n16, max_words, block_k, hilo));
}

cudaError_t launch_field_sampler(const SampleArgs &a, int max_m, int max_n16, int max_words,
                                 int block_k, bool hilo, int32_t *status, long long dec_wait_polls,
                                 cudaStream_t st) {
    // At most 512 / cols CTAs may share an SM (TMEM), and at most two by the registers of the
    // launch; the shared-memory request is raised so that no more than that fit on one SM (a
    // CTA's TMEM allocation would otherwise wait for another CTA's release).
    FieldLaunch L;
    L.cols = field_tmem_cols(max_n16, field_dcols(block_k, hilo));
    L.max_n16 = max_n16;
    L.ring = field_ring(max_n16, max_words, block_k, hilo);
    L.xs_chunks = field_xs_chunks(max_n16, field_dcols(block_k, hilo));
    const size_t per_sm = 228 * 1024, max_ctas = std::min<size_t>(2, 512 / L.cols);
    L.smem = field_smem_bytes(max_n16, max_words, block_k, hilo);
    const size_t floor_smem = per_sm / (max_ctas + 1) + 1;
    if (L.smem < floor_smem) L.smem = floor_smem;
    const long long polls = dec_wait_polls > 0 ? dec_wait_polls : 0;
    const bool track = a.run_cost != nullptr;
    if (block_k != 16)
        return launch_field_wide(a, max_m, block_k, hilo, track, status, polls, L, st);
    if (hilo)
        return track ? field_launch_mc<16, true, true>(a, max_m, status, polls, L, st)
                     : field_launch_mc<16, true, false>(a, max_m, status, polls, L, st);
    return track ? field_launch_mc<16, false, true>(a, max_m, status, polls, L, st)
                 : field_launch_mc<16, false, false>(a, max_m, status, polls, L, st);
}

}  // namespace sais
