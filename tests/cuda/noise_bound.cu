// Exhaustive check of the p-bit noise transform on the device (test program).
//
// The noise rho = (2v+1)/2^24 - 1 takes 2^24 values (v = word >> 8).  For every one of them this
// program compares the sampler's theta_of_word() with FP64 atanh(rho) and checks the error
// bound the samplers use in their decision guard, |theta - atanh(rho)| <= kThetaAbsErr +
// kThetaRelErr |theta|; it also checks that rho_of_word() is exact.  Prints one line:
//   values=<n> violations=<n> max_abs_err=<e> max_ratio=<r> rho_inexact=<n>
// (ratio = error / bound, must stay below 1).
#include <cstdio>

#include "sais_device.cuh"

using namespace sais;

__device__ unsigned long long d_viol, d_rho_bad;
__device__ unsigned int d_max_err_bits, d_max_ratio_bits;

__global__ void check(uint32_t nvals) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nvals; v += gridDim.x * blockDim.x) {
        const uint32_t w = v << 8;
        const float th = theta_of_word(w);
        const double rho = ((double)(2u * v + 1u) - 16777216.0) / 16777216.0;
        if ((double)rho_of_word(w) != rho) atomicAdd(&d_rho_bad, 1ull);
        const double ex = atanh(rho);
        const double err = fabs((double)th - ex);
        const double bound = (double)kThetaAbsErr + (double)kThetaRelErr * fabs((double)th);
        if (!(err <= bound)) atomicAdd(&d_viol, 1ull);
        const float ef = (float)err, rf = (float)(err / bound);
        atomicMax(&d_max_err_bits, __float_as_uint(ef));
        atomicMax(&d_max_ratio_bits, __float_as_uint(rf));
    }
}

int main() {
    const uint32_t n = 1u << 24;
    check<<<4096, 256>>>(n);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        printf("cuda error %s\n", cudaGetErrorString(e));
        return 2;
    }
    unsigned long long viol = 0, rbad = 0;
    unsigned int eb = 0, rb = 0;
    cudaMemcpyFromSymbol(&viol, d_viol, 8);
    cudaMemcpyFromSymbol(&rbad, d_rho_bad, 8);
    cudaMemcpyFromSymbol(&eb, d_max_err_bits, 4);
    cudaMemcpyFromSymbol(&rb, d_max_ratio_bits, 4);
    float me, mr;
    memcpy(&me, &eb, 4);
    memcpy(&mr, &rb, 4);
    printf("values=%u violations=%llu max_abs_err=%.6e max_ratio=%.4f rho_inexact=%llu\n", n, viol,
           (double)me, (double)mr, rbad);
    return (viol == 0 && rbad == 0) ? 0 : 1;
}
