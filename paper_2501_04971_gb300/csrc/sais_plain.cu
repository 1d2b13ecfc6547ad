// sais_plain.cu -- launch of the plain per-spin p-bit sampler (Sec. III-B, Eq. 9-10): one CTA of
// `chains_per_cta` threads per work item; the sampler itself is plain_item in
// sais_plain_item.cuh.
#include "sais_plain_item.cuh"

namespace sais {
namespace {

template <int MC, bool kF16>
__global__ void __launch_bounds__(128) plain_sampler_kernel(SampleArgs a) {
    const int j = a.work ? a.work[2 * blockIdx.x] : (int)blockIdx.y;
    const int grp = a.work ? a.work[2 * blockIdx.x + 1] : (int)blockIdx.x;
    plain_item<MC, kF16>(a, j, grp, (int)blockDim.x, (int)threadIdx.x);
}

template <int MC, bool kF16>
cudaError_t launch_mc(const SampleArgs &a, int cpb, size_t smem, cudaStream_t s) {
    auto kern = plain_sampler_kernel<MC, kF16>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid = a.work ? dim3(a.nwork, 1) : dim3((a.chains + cpb - 1) / cpb, a.count);
    kern<<<grid, cpb, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t plain_smem_bytes(int max_npad, int max_words, bool any_w, int cpb, bool f16) {
    return (any_w ? (size_t)max_npad * cpb * (f16 ? 2 : 4) : 0) + (size_t)max_words * cpb * 4;
}

template <bool kF16>
cudaError_t launch_f(const SampleArgs &a, int max_m, int cpb, size_t smem, cudaStream_t stream) {
    if (max_m <= 1) return launch_mc<1, kF16>(a, cpb, smem, stream);
    if (max_m <= 2) return launch_mc<2, kF16>(a, cpb, smem, stream);
    if (max_m <= 4) return launch_mc<4, kF16>(a, cpb, smem, stream);
    if (max_m <= 8) return launch_mc<8, kF16>(a, cpb, smem, stream);
    if (max_m <= 16) return launch_mc<16, kF16>(a, cpb, smem, stream);
    return launch_mc<32, kF16>(a, cpb, smem, stream);
}

cudaError_t launch_plain_sampler(const SampleArgs &a, int max_m, int max_npad, int max_words,
                                 int cpb, cudaStream_t stream, bool f16) {
    const bool any_w = max_npad > 0;
    const size_t smem = plain_smem_bytes(max_npad, max_words, any_w, cpb, f16 && any_w);
    // int16 F only where there is an F (linear objectives keep one instantiation)
    if (f16 && any_w) return launch_f<true>(a, max_m, cpb, smem, stream);
    return launch_f<false>(a, max_m, cpb, smem, stream);
}

}  // namespace sais
