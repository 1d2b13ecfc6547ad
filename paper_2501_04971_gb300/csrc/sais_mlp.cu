// sais_mlp.cu -- learned warm start of the Lagrange multipliers: a 7 -> 128 -> 128 -> 1 ReLU
// network with BF16 weights and FP32 accumulation, its training (mean squared error, Adam) and
// its inference, on the sm_103a tensor cores.  The paper has no learned part; the network maps
// per-constraint features of an instance to the multiplier the method converges to, so that
// Algorithm 1 can start from it instead of lambda = 0.
//
// Parameters (FP32 master copy, flat, kParams floats):
//   W1  [128 x 16]  at 0      column 7 = b1 (the input carries a constant 1 there), 8..15 zero
//   W2  [128 x 144] at 2048   column 128 = b2 (h1 carries a constant 1 there), 129..143 zero
//   w3  [128]       at 20480, b3 at 20608, three unused floats.
// Features x (rows x 8 floats, column 7 unused) are standardised in the kernel,
// x'_f = (x_f - mu_f) / sd_f, and the output is lambda = y_mu + y_sd * u.
//
// Training kernel, one CTA per 128 rows (M = 128 = TMEM lanes, thread s = row s):
//   Z1  = X' W1^T       1 MMA   (K = 16)            TMEM columns   0..127
//   Z2  = H1 W2^T       9 MMAs  (K = 144)           TMEM columns 128..255
//   u   = w3 . relu(Z2) + b3 on the CUDA cores; du = 2 (u - t') / B
//   dZ2 = du w3 * [Z2 > 0] (BF16)
//   dH1 = dZ2 W2        8 MMAs  (K = 128)           TMEM columns   0..127 (Z1 is consumed)
//   dW2 = dZ2^T [H1|1]  8 MMAs  (K = 128 rows, N = 144; column 128 = db2)   columns 256..399
//   dZ1 = dH1 * [Z1 > 0] (BF16)
//   dW1 = dZ1^T [X'|1]  8 MMAs  (N = 16; column 7 = db1)                  columns 448..463
//   dw3, db3 and the loss by warp reductions.
// Operands sit in shared memory in the no-swizzle K-major core-matrix layout: element (r, k) of
// an R x K operand at byte ((k/8)(R/8) + r/8) 128 + (r%8) 16 + (k%8) 2, so the leading byte
// offset (next core matrix along K) is 16 R and the stride byte offset (next 8 rows) is 128.
// The weights arrive as prebuilt BF16 images of that layout by three bulk copies (TMA engine).
// Each CTA writes its partial gradient; a second kernel sums the partials in CTA order
// (deterministic), applies Adam and republishes the BF16 images.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "sais_internal.h"
#include "sais_tc.cuh"

namespace sais {
namespace {

constexpr int kH = 128, kNF = 7, kK1 = 16, kK2 = 144, kRows = 128, kThreads = 128;
constexpr int kOffW1 = 0, kOffW2 = 2048, kOffW3 = 20480, kOffB3 = 20608;
constexpr int kParams = SAIS_MLP_PARAMS;
static_assert(kParams == 20612, "parameter layout");

// BF16 images (byte offsets inside the image buffer).
constexpr int kImgW1 = 0, kImgW1Bytes = kH * kK1 * 2;             // B of layer 1: 128 x 16
constexpr int kImgW2 = 4096, kImgW2Bytes = kH * kK2 * 2;          // B of layer 2: 128 x 144
constexpr int kImgW2T = 40960, kImgW2TBytes = kH * kH * 2;        // B of dH1: W2^T, 128 x 128
constexpr int kImgW3 = 73728;                                     // w3[128], b3 (BF16)
constexpr int kImgBytes = 73984;

// Shared-memory map of the training / inference kernel.
constexpr int kSmXA = 0;          // X' as A (128 x 16)
constexpr int kSmXT = 4096;       // [X'|1]^T as B of dW1 (16 x 128)
constexpr int kSmW1 = 8192;       // W1 image
constexpr int kSmW2 = 12288;      // W2 image; later dZ2^T as A of dW2 (128 x 128)
constexpr int kSmW2T = 49152;     // W2^T image; later dZ1^T as A of dW1 (128 x 128)
constexpr int kSmH1 = 81920;      // [H1|1] as A of layer 2 (128 x 144); later dZ2 as A of dH1
constexpr int kSmH1T = 118784;    // [H1|1]^T as B of dW2 (144 x 128)
constexpr int kSmW3 = 155648;     // w3, b3 as FP32 (129)
constexpr int kSmRed = 156672;    // [4 warps][128] column partial sums of dw3
constexpr int kSmMisc = 158720;   // per-warp loss and db3 partials
constexpr int kSmBar = 158784;    // 2 mbarriers
constexpr int kSmTmem = 158800;   // TMEM base address slot
constexpr int kSmBytes = 158848;

constexpr uint32_t kColZ1 = 0, kColZ2 = 128, kColDW2 = 256, kColDW1 = 448, kTmemCols = 512;
constexpr long long kWaitCycles = 4000000000LL;

__host__ __device__ constexpr uint32_t core_off(uint32_t r, uint32_t k, uint32_t R) {
    return ((k >> 3) * (R >> 3) + (r >> 3)) * 128u + (r & 7u) * 16u + (k & 7u) * 2u;
}

__device__ __forceinline__ uint16_t bf16_bits(float f) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}
__device__ __forceinline__ float bf16_float(uint16_t b) {
    return __bfloat162float(__ushort_as_bfloat16(b));
}
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    return (uint32_t)bf16_bits(lo) | ((uint32_t)bf16_bits(hi) << 16);
}

struct MlpNorm {
    float mu[kNF], sd[kNF], y_mu, y_sd;
};

struct MlpArgs {
    const float *X;          // rows x 8
    const float *target;     // rows (training) or NULL
    int32_t rows;
    float inv_rows;          // 1 / rows
    MlpNorm norm;
    const uint16_t *img;     // BF16 images
    float *y;                // inference: lambda per row, or NULL
    float *lam;              // warm start: lambda array, or NULL
    const int32_t *dst;      // warm start: row -> index into lam
    float *part;             // training: [gridDim.x][kParams] partial gradients
    int32_t *status;         // device status word or NULL
};

__device__ bool wait_bar(uint64_t *bar, uint32_t parity, int32_t *status) {
    const long long t0 = clock64();
    while (!tc::mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) {
            if (status) atomicExch(status, (int32_t)SAIS_ETIMEOUT);
            return false;
        }
    }
    return true;
}

// Column sums over the 32 lanes of v[0..31] (lane L ends with the sum of column L in v[0]):
// a butterfly that halves the kept columns at every step, summing in a fixed order.
__device__ __forceinline__ float warp_colsum32(float (&v)[32], int lane) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const float send = upper ? v[i] : v[i + off];
            const float keep = upper ? v[i + off] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return v[0];
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

template <bool kTrain>
__global__ void __launch_bounds__(kThreads, 1) mlp_kernel(MlpArgs a) {
    extern __shared__ __align__(128) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = blockIdx.x * kRows + tid;
    const bool valid = row < a.rows;
    uint64_t *bar_w = reinterpret_cast<uint64_t *>(sm + kSmBar);
    uint64_t *bar_mma = bar_w + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + kSmTmem);
    float *w3s = reinterpret_cast<float *>(sm + kSmW3);
    float *red = reinterpret_cast<float *>(sm + kSmRed);
    float *misc = reinterpret_cast<float *>(sm + kSmMisc);
    const uint32_t sbase = tc::smem_u32(sm);

    if (warp == 0) {
        tc::tmem_alloc(tslot, kTmemCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(bar_w, 1);
        tc::mbar_init(bar_mma, 1);
        tc::fence_mbar_init();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        const unsigned char *img = reinterpret_cast<const unsigned char *>(a.img);
        tc::mbar_expect_tx(bar_w, kImgW1Bytes + kImgW2Bytes + (kTrain ? kImgW2TBytes : 0));
        tc::bulk_g2s(sm + kSmW1, img + kImgW1, kImgW1Bytes, bar_w);
        tc::bulk_g2s(sm + kSmW2, img + kImgW2, kImgW2Bytes, bar_w);
        if (kTrain) tc::bulk_g2s(sm + kSmW2T, img + kImgW2T, kImgW2TBytes, bar_w);
    }
    w3s[tid] = bf16_float(a.img[kImgW3 / 2 + tid]);
    if (tid == 0) w3s[kH] = bf16_float(a.img[kImgW3 / 2 + kH]);

    // Standardised features, the bias input 1 at column 7, zero padding to K = 16.
    float xp[kK1];
    {
        float xr[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (valid) {
            const float4 *src = reinterpret_cast<const float4 *>(a.X + (size_t)row * 8);
            const float4 v0 = src[0], v1 = src[1];
            xr[0] = v0.x; xr[1] = v0.y; xr[2] = v0.z; xr[3] = v0.w;
            xr[4] = v1.x; xr[5] = v1.y; xr[6] = v1.z;
        }
#pragma unroll
        for (int f = 0; f < kK1; ++f)
            xp[f] = f < kNF ? (valid ? (xr[f] - a.norm.mu[f]) / a.norm.sd[f] : 0.f)
                            : (f == kNF ? 1.f : 0.f);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        uint4 v;
        v.x = pack2(xp[8 * q + 0], xp[8 * q + 1]);
        v.y = pack2(xp[8 * q + 2], xp[8 * q + 3]);
        v.z = pack2(xp[8 * q + 4], xp[8 * q + 5]);
        v.w = pack2(xp[8 * q + 6], xp[8 * q + 7]);
        *reinterpret_cast<uint4 *>(sm + kSmXA + core_off(tid, 8 * q, kRows)) = v;
    }
    // [H1|1]: columns 128..143 of row s hold 1, 0, ..., 0
    *reinterpret_cast<uint4 *>(sm + kSmH1 + core_off(tid, 128, kRows)) =
        make_uint4(pack2(1.f, 0.f), 0u, 0u, 0u);
    *reinterpret_cast<uint4 *>(sm + kSmH1 + core_off(tid, 136, kRows)) = make_uint4(0u, 0u, 0u, 0u);
    if (kTrain) {
#pragma unroll
        for (int f = 0; f < kK1; ++f)
            *reinterpret_cast<uint16_t *>(sm + kSmXT + core_off(f, tid, kK1)) =
                bf16_bits(f == kNF ? 1.f : xp[f]);
#pragma unroll
        for (int r = kH; r < kK2; ++r)
            *reinterpret_cast<uint16_t *>(sm + kSmH1T + core_off(r, tid, kK2)) =
                bf16_bits(r == kH ? 1.f : 0.f);
    }
    tc::fence_proxy_async_smem();
    __syncthreads();

    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    uint32_t mma_phase = 0;
    bool ok = true;

    // ---- layer 1: Z1 = X' W1^T ----------------------------------------------------------------
    if (tid == 0) {
        if (wait_bar(bar_w, 0, a.status)) {
            tc::tc_fence_after();
            tc::mma_bf16(tmem + kColZ1, tc::smem_desc(sbase + kSmXA, 16 * kRows, 128),
                         tc::smem_desc(sbase + kSmW1, 16 * kH, 128), tc::idesc_bf16_f32(128, 128),
                         0u);
        }
        tc::mma_commit(bar_mma);
    }
    ok = wait_bar(bar_mma, mma_phase, a.status) && ok;
    mma_phase ^= 1u;
    tc::tc_fence_after();

    // ReLU, mask, [H1|1] (and its transpose for dW2)
    uint32_t m1[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float z[32];
        tc::tmem_ld32(tmem + lane_base + kColZ1 + 32 * c, z);
        uint32_t mb = 0u;
#pragma unroll
        for (int e = 0; e < 32; ++e) {
            if (z[e] > 0.f) mb |= 1u << e;
            z[e] = fmaxf(z[e], 0.f);
        }
        m1[c] = mb;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float *zz = z + 8 * q;
            *reinterpret_cast<uint4 *>(sm + kSmH1 + core_off(tid, 32 * c + 8 * q, kRows)) =
                make_uint4(pack2(zz[0], zz[1]), pack2(zz[2], zz[3]), pack2(zz[4], zz[5]),
                           pack2(zz[6], zz[7]));
        }
        if (kTrain) {
#pragma unroll
            for (int e = 0; e < 32; ++e)
                *reinterpret_cast<uint16_t *>(sm + kSmH1T + core_off(32 * c + e, tid, kK2)) =
                    bf16_bits(z[e]);
        }
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();

    // ---- layer 2: Z2 = [H1|1] W2^T ----------------------------------------------------------
    if (tid == 0) {
        tc::tc_fence_after();
#pragma unroll 1
        for (int kk = 0; kk < kK2 / 16; ++kk)
            tc::mma_bf16(tmem + kColZ2,
                         tc::smem_desc(sbase + kSmH1 + kk * 2 * (kRows / 8) * 128, 16 * kRows, 128),
                         tc::smem_desc(sbase + kSmW2 + kk * 2 * (kH / 8) * 128, 16 * kH, 128),
                         tc::idesc_bf16_f32(128, 128), kk > 0 ? 1u : 0u);
        tc::mma_commit(bar_mma);
    }
    ok = wait_bar(bar_mma, mma_phase, a.status) && ok;
    mma_phase ^= 1u;
    tc::tc_fence_after();

    float u = w3s[kH];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float z[32];
        tc::tmem_ld32(tmem + lane_base + kColZ2 + 32 * c, z);
#pragma unroll
        for (int e = 0; e < 32; ++e) u = fmaf(w3s[32 * c + e], fmaxf(z[e], 0.f), u);
    }

    if (!kTrain) {
        if (valid) {
            const float val = fmaf(a.norm.y_sd, u, a.norm.y_mu);
            if (a.y) a.y[row] = val;
            if (a.lam) a.lam[a.dst[row]] = fmaxf(val, 0.f);
        }
    } else {
        float e = 0.f, du = 0.f;
        if (valid) {
            const float tn = (a.target[row] - a.norm.y_mu) / a.norm.y_sd;
            e = u - tn;
            du = 2.f * e * a.inv_rows;
        }
        const float le = warp_sum(e * e), ld = warp_sum(du);
        if (lane == 0) {
            misc[warp] = le;
            misc[4 + warp] = ld;
        }
        // dw3 partial column sums, and dZ2 = du w3 [Z2 > 0] into dZ2 (A of dH1) and dZ2^T
        // (A of dW2); both regions were read by the layer-2 MMAs, which have completed.
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float z[32], v[32];
            tc::tmem_ld32(tmem + lane_base + kColZ2 + 32 * c, z);
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                v[q] = du * fmaxf(z[q], 0.f);
                z[q] = z[q] > 0.f ? du * w3s[32 * c + q] : 0.f;
            }
            const float cs = warp_colsum32(v, lane);
            red[warp * kH + 32 * c + lane] = cs;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float *zz = z + 8 * q;
                *reinterpret_cast<uint4 *>(sm + kSmH1 + core_off(tid, 32 * c + 8 * q, kRows)) =
                    make_uint4(pack2(zz[0], zz[1]), pack2(zz[2], zz[3]), pack2(zz[4], zz[5]),
                               pack2(zz[6], zz[7]));
            }
#pragma unroll
            for (int q = 0; q < 32; ++q)
                *reinterpret_cast<uint16_t *>(sm + kSmW2 + core_off(32 * c + q, tid, kH)) =
                    bf16_bits(z[q]);
        }
        tc::fence_proxy_async_smem();
        tc::tc_fence_before();
        __syncthreads();

        float *part = a.part + (size_t)blockIdx.x * kParams;
        part[kOffW3 + tid] = ((red[tid] + red[kH + tid]) + red[2 * kH + tid]) + red[3 * kH + tid];
        if (tid == 0) {
            part[kOffB3] = ((misc[4] + misc[5]) + misc[6]) + misc[7];
            part[kOffB3 + 1] = ((misc[0] + misc[1]) + misc[2]) + misc[3];   // loss partial
        }

        // ---- dH1 = dZ2 W2 and dW2 = dZ2^T [H1|1] -----------------------------------------
        if (tid == 0) {
            tc::tc_fence_after();
#pragma unroll 1
            for (int kk = 0; kk < kH / 16; ++kk)
                tc::mma_bf16(tmem + kColZ1,
                             tc::smem_desc(sbase + kSmH1 + kk * 2 * (kRows / 8) * 128, 16 * kRows,
                                           128),
                             tc::smem_desc(sbase + kSmW2T + kk * 2 * (kH / 8) * 128, 16 * kH, 128),
                             tc::idesc_bf16_f32(128, 128), kk > 0 ? 1u : 0u);
#pragma unroll 1
            for (int kk = 0; kk < kRows / 16; ++kk)
                tc::mma_bf16(tmem + kColDW2,
                             tc::smem_desc(sbase + kSmW2 + kk * 2 * (kH / 8) * 128, 16 * kH, 128),
                             tc::smem_desc(sbase + kSmH1T + kk * 2 * (kK2 / 8) * 128, 16 * kK2,
                                           128),
                             tc::idesc_bf16_f32(128, kK2), kk > 0 ? 1u : 0u);
            tc::mma_commit(bar_mma);
        }
        ok = wait_bar(bar_mma, mma_phase, a.status) && ok;
        mma_phase ^= 1u;
        tc::tc_fence_after();

        // dZ1 = dH1 [Z1 > 0] as dZ1^T (A of dW1) into the W2^T region (read by the dH1 MMAs)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float d[32];
            tc::tmem_ld32(tmem + lane_base + kColZ1 + 32 * c, d);
#pragma unroll
            for (int q = 0; q < 32; ++q)
                *reinterpret_cast<uint16_t *>(sm + kSmW2T + core_off(32 * c + q, tid, kH)) =
                    bf16_bits(((m1[c] >> q) & 1u) ? d[q] : 0.f);
        }
        // row `tid` of dW2 (output unit o = tid), stored column-major so that stores coalesce
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float g[32];
            tc::tmem_ld32(tmem + lane_base + kColDW2 + 32 * c, g);
#pragma unroll
            for (int q = 0; q < 32; ++q) part[kOffW2 + (32 * c + q) * kH + tid] = g[q];
        }
        {
            float g[16];
            tc::tmem_ld16(tmem + lane_base + kColDW2 + 128, g);
#pragma unroll
            for (int q = 0; q < 16; ++q) part[kOffW2 + (128 + q) * kH + tid] = g[q];
        }
        tc::fence_proxy_async_smem();
        tc::tc_fence_before();
        __syncthreads();

        // ---- dW1 = dZ1^T [X'|1] -----------------------------------------------------------
        if (tid == 0) {
            tc::tc_fence_after();
#pragma unroll 1
            for (int kk = 0; kk < kRows / 16; ++kk)
                tc::mma_bf16(tmem + kColDW1,
                             tc::smem_desc(sbase + kSmW2T + kk * 2 * (kH / 8) * 128, 16 * kH, 128),
                             tc::smem_desc(sbase + kSmXT + kk * 2 * (kK1 / 8) * 128, 16 * kK1, 128),
                             tc::idesc_bf16_f32(128, kK1), kk > 0 ? 1u : 0u);
            tc::mma_commit(bar_mma);
        }
        ok = wait_bar(bar_mma, mma_phase, a.status) && ok;
        mma_phase ^= 1u;
        tc::tc_fence_after();
        {
            float g[16];
            tc::tmem_ld16(tmem + lane_base + kColDW1, g);
#pragma unroll
            for (int q = 0; q < 16; ++q) part[kOffW1 + q * kH + tid] = g[q];
        }
    }

    // Teardown: the weight copies must have landed before the CTA exits (bounded).
    if (tid == 0 && !ok) wait_bar(bar_w, 0, a.status);
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

// Sum of the per-CTA partials (in CTA order), then: mode 0 writes the gradient, mode 1 takes an
// Adam step; modes 1 and 2 publish the BF16 images of the (new) parameters.
struct UpdateArgs {
    int mode;
    const float *part;
    int32_t nparts;
    float inv_rows;
    float *grad;
    float *theta, *mom, *vel;
    float lr, b1, b2, eps, c1, c2;   // c1 = 1 - b1^t, c2 = 1 - b2^t
    uint16_t *img;
    float *loss;
};

__global__ void mlp_update_kernel(UpdateArgs u) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kParams;
         p += gridDim.x * blockDim.x) {
        if (p > kOffB3) {   // unused tail of the parameter vector: zero gradient, no update
            if (u.mode == 0) u.grad[p] = 0.f;
            continue;
        }
        int pi = p, o = 0, k = 0, blk = 2;
        if (p < kOffW2) {
            o = p / kK1;
            k = p % kK1;
            pi = kOffW1 + k * kH + o;
            blk = 0;
        } else if (p < kOffW3) {
            o = (p - kOffW2) / kK2;
            k = (p - kOffW2) % kK2;
            pi = kOffW2 + k * kH + o;
            blk = 1;
        }
        float th = u.theta[p];
        if (u.mode != 2) {
            float g = 0.f;
            for (int c = 0; c < u.nparts; ++c) g += u.part[(size_t)c * kParams + pi];
            if (u.mode == 0) {
                u.grad[p] = g;
                continue;
            }
            const float m = u.b1 * u.mom[p] + (1.f - u.b1) * g;
            const float v = u.b2 * u.vel[p] + (1.f - u.b2) * g * g;
            u.mom[p] = m;
            u.vel[p] = v;
            th -= u.lr * (m / u.c1) / (sqrtf(v / u.c2) + u.eps);
            u.theta[p] = th;
        }
        const uint16_t b = bf16_bits(th);
        if (blk == 0) {
            u.img[(kImgW1 + core_off(o, k, kH)) / 2] = b;
        } else if (blk == 1) {
            u.img[(kImgW2 + core_off(o, k, kH)) / 2] = b;
            if (k < kH) u.img[(kImgW2T + core_off(k, o, kH)) / 2] = b;
        } else {
            u.img[kImgW3 / 2 + (p - kOffW3)] = b;
        }
    }
    if (u.mode != 2 && u.loss && blockIdx.x == 0 && threadIdx.x == 0) {
        float s = 0.f;
        for (int c = 0; c < u.nparts; ++c) s += u.part[(size_t)c * kParams + kOffB3 + 1];
        *u.loss = s * u.inv_rows;
    }
}

}  // namespace
}  // namespace sais

using namespace sais;

struct sais_mlp {
    int device = 0;
    float *theta = nullptr, *mom = nullptr, *vel = nullptr;   // FP32 master, Adam moments
    uint16_t *img = nullptr;                                  // BF16 images
    float *part = nullptr;                                    // per-CTA partial gradients
    int32_t part_cap = 0;
    int32_t *status = nullptr;
    int32_t step = 0;
    MlpNorm norm{};
};

namespace {

struct Guard {
    int prev = 0;
    explicit Guard(int dev) {
        cudaGetDevice(&prev);
        cudaSetDevice(dev);
    }
    ~Guard() { cudaSetDevice(prev); }
};

uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

sais_status mlp_launch_update(sais_mlp *m, int mode, int nparts, float inv_rows, float *grad,
                              float lr, float *loss, cudaStream_t st) {
    UpdateArgs u{};
    u.mode = mode;
    u.part = m->part;
    u.nparts = nparts;
    u.inv_rows = inv_rows;
    u.grad = grad;
    u.theta = m->theta;
    u.mom = m->mom;
    u.vel = m->vel;
    u.img = m->img;
    u.loss = loss;
    if (mode == 1) {
        const int t = m->step + 1;
        u.lr = lr;
        u.b1 = 0.9f;
        u.b2 = 0.999f;
        u.eps = 1e-8f;
        // bias corrections from the FP32 betas the kernel uses (at t = 1 they cancel exactly)
        u.c1 = (float)(1.0 - std::pow((double)u.b1, t));
        u.c2 = (float)(1.0 - std::pow((double)u.b2, t));
    }
    mlp_update_kernel<<<(kParams + 255) / 256, 256, 0, st>>>(u);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(SAIS_ECUDA, "MLP update launch: %s", cudaGetErrorString(e));
    if (mode == 1) ++m->step;
    return SAIS_OK;
}

sais_status mlp_launch(const sais_mlp *m, bool train, const float *X, const float *t,
                       int32_t rows, float *y, float *lam, const int32_t *dst, cudaStream_t st) {
    MlpArgs a{};
    a.X = X;
    a.target = t;
    a.rows = rows;
    a.inv_rows = 1.f / (float)rows;
    a.norm = m->norm;
    a.img = m->img;
    a.y = y;
    a.lam = lam;
    a.dst = dst;
    a.part = m->part;
    a.status = m->status;
    auto kern = train ? mlp_kernel<true> : mlp_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmBytes);
    if (e == cudaSuccess) {
        kern<<<(rows + kRows - 1) / kRows, kThreads, kSmBytes, st>>>(a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return set_error(SAIS_ECUDA, "MLP launch: %s", cudaGetErrorString(e));
    return SAIS_OK;
}

sais_status ensure_parts(sais_mlp *m, int32_t rows) {
    const int32_t need = (rows + kRows - 1) / kRows;
    if (need <= m->part_cap) return SAIS_OK;
    if (m->part) {
        cudaDeviceSynchronize();   // queued launches may still write the old partials
        dev_free(m->part);
    }
    m->part = nullptr;
    m->part_cap = 0;
    cudaError_t e = dev_alloc(reinterpret_cast<void **>(&m->part),
                              (size_t)need * kParams * sizeof(float));
    if (e != cudaSuccess) return set_error(SAIS_ENOMEM, "MLP partial gradients: %s", cudaGetErrorString(e));
    m->part_cap = need;
    return SAIS_OK;
}

bool check_x(const sais_mlp *m, const void *X, int32_t rows) {
    return m && X && rows >= 1;
}

}  // namespace

extern "C" {

sais_status sais_mlp_create(int32_t device, uint64_t seed, sais_mlp **out) {
    if (!out) return set_error(SAIS_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return set_error(SAIS_EINVAL, "device %d not available", device);
    Guard g(device);
    sais_mlp *m = new (std::nothrow) sais_mlp;
    if (!m) return set_error(SAIS_ENOMEM, "host allocation failed");
    m->device = device;
    cudaError_t e = dev_alloc(reinterpret_cast<void **>(&m->theta), kParams * sizeof(float) * 3);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&m->img), kImgBytes);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&m->status), sizeof(int32_t));
    if (e != cudaSuccess) {
        sais_mlp_destroy(m);
        return set_error(SAIS_ENOMEM, "MLP buffers: %s", cudaGetErrorString(e));
    }
    m->mom = m->theta + kParams;
    m->vel = m->theta + 2 * kParams;
    cudaMemset(m->img, 0, kImgBytes);
    cudaMemset(m->status, 0, sizeof(int32_t));
    // He-uniform hidden layers, a smaller uniform output layer, zero biases.
    std::vector<float> p(kParams, 0.f);
    uint64_t s = seed;
    auto uni = [&](double bound) {
        return (float)(bound * (2.0 * ((splitmix64(s) >> 11) * 0x1.0p-53) - 1.0));
    };
    for (int o = 0; o < kH; ++o)
        for (int k = 0; k < kNF; ++k) p[kOffW1 + o * kK1 + k] = uni(std::sqrt(6.0 / kNF));
    for (int o = 0; o < kH; ++o)
        for (int k = 0; k < kH; ++k) p[kOffW2 + o * kK2 + k] = uni(std::sqrt(6.0 / kH));
    for (int o = 0; o < kH; ++o) p[kOffW3 + o] = uni(std::sqrt(3.0 / kH));
    float nrm[16];
    for (int f = 0; f < kNF; ++f) {
        nrm[f] = 0.f;
        nrm[kNF + f] = 1.f;
    }
    nrm[14] = 0.f;
    nrm[15] = 1.f;
    sais_status st = sais_mlp_set_params(m, p.data(), nrm);
    if (st != SAIS_OK) {
        sais_mlp_destroy(m);
        return st;
    }
    *out = m;
    return SAIS_OK;
}

sais_status sais_mlp_destroy(sais_mlp *m) {
    if (!m) return SAIS_OK;
    Guard g(m->device);
    cudaDeviceSynchronize();   // the handle's queued launches finish before its buffers go
    dev_free(m->theta);
    dev_free(m->img);
    dev_free(m->part);
    dev_free(m->status);
    delete m;
    return SAIS_OK;
}

sais_status sais_mlp_set_params(sais_mlp *m, const float *params, const float *norm) {
    if (!m || !params) return set_error(SAIS_EINVAL, "NULL argument");
    std::vector<float> p(params, params + kParams);
    for (int o = 0; o < kH; ++o) {
        for (int k = kNF + 1; k < kK1; ++k) p[kOffW1 + o * kK1 + k] = 0.f;
        for (int k = kH + 1; k < kK2; ++k) p[kOffW2 + o * kK2 + k] = 0.f;
    }
    for (int i = kOffB3 + 1; i < kParams; ++i) p[i] = 0.f;
    if (norm) {
        for (int f = 0; f < kNF; ++f)
            if (!(norm[kNF + f] > 0.f) || !std::isfinite(norm[f]) || !std::isfinite(norm[kNF + f]))
                return set_error(SAIS_EINVAL, "norm: sd[%d] must be finite and > 0", f);
        if (!(norm[15] > 0.f) || !std::isfinite(norm[14]) || !std::isfinite(norm[15]))
            return set_error(SAIS_EINVAL, "norm: y_sd must be finite and > 0");
        for (int f = 0; f < kNF; ++f) {
            m->norm.mu[f] = norm[f];
            m->norm.sd[f] = norm[kNF + f];
        }
        m->norm.y_mu = norm[14];
        m->norm.y_sd = norm[15];
    }
    Guard g(m->device);
    cudaError_t e = cudaMemcpy(m->theta, p.data(), kParams * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->mom, 0, 2 * kParams * sizeof(float));
    if (e != cudaSuccess) return set_error(SAIS_ECUDA, "MLP parameters: %s", cudaGetErrorString(e));
    m->step = 0;
    sais_status s = mlp_launch_update(m, 2, 0, 0.f, nullptr, 0.f, nullptr, 0);
    if (s != SAIS_OK) return s;
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return set_error(SAIS_ECUDA, "MLP publish: %s", cudaGetErrorString(e));
    return SAIS_OK;
}

sais_status sais_mlp_get_params(const sais_mlp *m, float *params, float *norm) {
    if (!m) return set_error(SAIS_EINVAL, "NULL argument");
    Guard g(m->device);
    if (params) {
        cudaError_t e = cudaMemcpy(params, m->theta, kParams * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return set_error(SAIS_ECUDA, "MLP parameters: %s", cudaGetErrorString(e));
    }
    if (norm) {
        for (int f = 0; f < kNF; ++f) {
            norm[f] = m->norm.mu[f];
            norm[kNF + f] = m->norm.sd[f];
        }
        norm[14] = m->norm.y_mu;
        norm[15] = m->norm.y_sd;
    }
    return SAIS_OK;
}

sais_status sais_mlp_fit_normalization(sais_mlp *m, const float *X, const float *y, int32_t rows) {
    if (!m || !X || !y || rows < 1) return set_error(SAIS_EINVAL, "NULL argument or rows < 1");
    double s[kNF + 1] = {0}, ss[kNF + 1] = {0};
    for (int r = 0; r < rows; ++r)
        for (int f = 0; f <= kNF; ++f) {
            const double v = f < kNF ? (double)X[(size_t)r * 8 + f] : (double)y[r];
            s[f] += v;
            ss[f] += v * v;
        }
    float nrm[16];
    for (int f = 0; f <= kNF; ++f) {
        const double mu = s[f] / rows, var = ss[f] / rows - mu * mu;
        const double sd = var > 1e-12 ? std::sqrt(var) : 1.0;
        if (f < kNF) {
            nrm[f] = (float)mu;
            nrm[kNF + f] = (float)sd;
        } else {
            nrm[14] = (float)mu;
            nrm[15] = (float)sd;
        }
    }
    for (int f = 0; f < kNF; ++f) {
        m->norm.mu[f] = nrm[f];
        m->norm.sd[f] = nrm[kNF + f];
    }
    m->norm.y_mu = nrm[14];
    m->norm.y_sd = nrm[15];
    return SAIS_OK;
}

sais_status sais_mlp_forward(const sais_mlp *m, const float *X, int32_t rows, float *y,
                             void *stream) {
    if (!check_x(m, X, rows) || !y) return set_error(SAIS_EINVAL, "NULL argument or rows < 1");
    Guard g(m->device);
    return mlp_launch(m, false, X, nullptr, rows, y, nullptr, nullptr,
                      static_cast<cudaStream_t>(stream));
}

sais_status sais_mlp_gradient(sais_mlp *m, const float *X, const float *t, int32_t rows,
                              float *grad, float *loss, void *stream) {
    if (!check_x(m, X, rows) || !t || !grad) return set_error(SAIS_EINVAL, "NULL argument or rows < 1");
    Guard g(m->device);
    sais_status s = ensure_parts(m, rows);
    if (s != SAIS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = mlp_launch(m, true, X, t, rows, nullptr, nullptr, nullptr, st);
    if (s != SAIS_OK) return s;
    return mlp_launch_update(m, 0, (rows + kRows - 1) / kRows, 1.f / (float)rows, grad, 0.f, loss, st);
}

sais_status sais_mlp_train_step(sais_mlp *m, const float *X, const float *t, int32_t rows,
                                float lr, float *loss, void *stream) {
    if (!check_x(m, X, rows) || !t) return set_error(SAIS_EINVAL, "NULL argument or rows < 1");
    if (!(lr > 0.f) || !std::isfinite(lr)) return set_error(SAIS_EINVAL, "lr must be finite and > 0");
    Guard g(m->device);
    sais_status s = ensure_parts(m, rows);
    if (s != SAIS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = mlp_launch(m, true, X, t, rows, nullptr, nullptr, nullptr, st);
    if (s != SAIS_OK) return s;
    return mlp_launch_update(m, 1, (rows + kRows - 1) / kRows, 1.f / (float)rows, nullptr, lr, loss, st);
}

sais_status sais_mlp_status(sais_mlp *m) {
    if (!m) return set_error(SAIS_EINVAL, "NULL argument");
    Guard g(m->device);
    int32_t v = 0;
    cudaError_t e = cudaMemcpy(&v, m->status, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_error(SAIS_ECUDA, "MLP status: %s", cudaGetErrorString(e));
    if (v != SAIS_OK) {
        cudaMemset(m->status, 0, 4);
        return set_error((sais_status)v, "an MLP kernel reported: %s", sais_status_string((sais_status)v));
    }
    return SAIS_OK;
}

}  // extern "C"

namespace sais {
sais_status mlp_warm_start_launch(const sais_mlp *m, const float *feat, const int32_t *dst,
                                  int32_t rows, float *lambda, int device, cudaStream_t st) {
    if (!m) return set_error(SAIS_EINVAL, "NULL MLP");
    if (m->device != device)
        return set_error(SAIS_EINVAL, "MLP on device %d, problem on device %d", m->device, device);
    if (rows == 0) return SAIS_OK;
    return mlp_launch(m, false, feat, nullptr, rows, nullptr, lambda, dst, st);
}
}  // namespace sais
