// sais_plain.cu -- launch of the plain per-spin p-bit sampler (Sec. III-B, Eq. 9-10): one CTA of
// `chains_per_cta` threads per work item; the sampler itself is plain_item in
// sais_plain_item.cuh.
#include "sais_plain_item.cuh"

namespace sais {
namespace {

template <int MC>
__global__ void __launch_bounds__(128) plain_sampler_kernel(SampleArgs a) {
    const int j = a.work ? a.work[2 * blockIdx.x] : (int)blockIdx.y;
    const int grp = a.work ? a.work[2 * blockIdx.x + 1] : (int)blockIdx.x;
    plain_item<MC>(a, j, grp, (int)blockDim.x, (int)threadIdx.x);
}

template <int MC>
cudaError_t launch_mc(const SampleArgs &a, int cpb, size_t smem, cudaStream_t s) {
    auto kern = plain_sampler_kernel<MC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid = a.work ? dim3(a.nwork, 1) : dim3((a.chains + cpb - 1) / cpb, a.count);
    kern<<<grid, cpb, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t plain_smem_bytes(int max_npad, int max_words, bool any_w, int cpb) {
    return (any_w ? (size_t)max_npad * cpb * 4 : 0) + (size_t)max_words * cpb * 4;
}

cudaError_t launch_plain_sampler(const SampleArgs &a, int max_m, int max_npad, int max_words,
                                 int cpb, cudaStream_t stream) {
    const bool any_w = max_npad > 0;
    const size_t smem = plain_smem_bytes(max_npad, max_words, any_w, cpb);
    if (max_m <= 1) return launch_mc<1>(a, cpb, smem, stream);
    if (max_m <= 2) return launch_mc<2>(a, cpb, smem, stream);
    if (max_m <= 4) return launch_mc<4>(a, cpb, smem, stream);
    if (max_m <= 8) return launch_mc<8>(a, cpb, smem, stream);
    if (max_m <= 16) return launch_mc<16>(a, cpb, smem, stream);
    return launch_mc<32>(a, cpb, smem, stream);
}

}  // namespace sais
