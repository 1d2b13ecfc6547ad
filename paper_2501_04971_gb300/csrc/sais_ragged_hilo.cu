// sais_ragged_hilo.cu -- the persistent ragged-batch kernel with the BF16 hi/lo split of W (pair
// values above 256); launch logic in sais_ragged.cu.
#include "sais_ragged_kernel.cuh"

namespace sais {

cudaError_t launch_ragged_hilo(const SampleArgs &a, const int32_t *items, int32_t nitems,
                               int32_t *head, unsigned long long *stats, const FieldLaunch &L,
                               int grid, int32_t *status, long long polls, cudaStream_t st) {
    return ragged_launch_h<true>(a, items, nitems, head, stats, L, grid, status, polls, st);
}

}  // namespace sais
