// sais_post.cu -- the CPU-side steps of Algorithm 1 done on the device, one CTA per instance:
//   "store feasible x_k" -> keep the best feasible sample (min cost; first achiever in
//                           (iteration, chain) order on ties), count feasible samples;
//   "lambda <- lambda + eta g(x_k)" -> exact int64 sum of g over the chains (warp shuffles),
//                           FP64 mean and step in a fixed order, optional projection on
//                           lambda >= 0, rounded to FP32.
#include <climits>

#include "sais_device.cuh"

namespace sais {
namespace {

constexpr int kPostThreads = 256;

__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Lexicographic min of (cost, chain) across the warp.
__device__ __forceinline__ void warp_argmin(long long &c, int &ch) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long oc = __shfl_xor_sync(0xffffffffu, c, o);
        const int och = __shfl_xor_sync(0xffffffffu, ch, o);
        if (oc < c || (oc == c && och < ch)) {
            c = oc;
            ch = och;
        }
    }
}

__global__ void __launch_bounds__(kPostThreads) post_kernel(PostArgs a) {
    const int j = blockIdx.x;
    const int m = a.inst[j].m;
    const int C = a.inst_chains ? a.inst_chains[j] : a.chains;   // this instance's chains
    const size_t base = (size_t)j * a.chains;                     // rows are strided by `chains`
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kWarps = kPostThreads / 32;
    const uint32_t iter = a.iter_dev ? *a.iter_dev : a.iter;

    __shared__ long long red[kWarps];
    __shared__ int redi[kWarps];
    __shared__ long long gsum[kMaxConstraints];
    __shared__ int s_best_chain;
    __shared__ int s_copy;

    // Sum over chains of g_k, exact in int64.
    for (int k = 0; k < (a.do_lambda ? m : 0); ++k) {
        long long s = 0;
        for (int c = tid; c < C; c += kPostThreads) s += a.g[(base + c) * a.m_stride + k];
        s = warp_sum(s);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (tid == 0) {
            long long t = 0;
            for (int w = 0; w < kWarps; ++w) t += red[w];
            gsum[k] = t;
        }
        __syncthreads();
    }

    if (a.track_best) {
        long long bc = LLONG_MAX;
        int bch = INT_MAX, nf = 0;
        for (int c = tid; c < C; c += kPostThreads) {
            // feasible == NULL: a sample is feasible iff its cost is set (best-in-run outputs)
            if (a.feasible ? a.feasible[base + c] != 0 : a.cost[base + c] != LLONG_MAX) {
                ++nf;
                const long long v = a.cost[base + c];
                if (v < bc || (v == bc && c < bch)) {
                    bc = v;
                    bch = c;
                }
            }
        }
        warp_argmin(bc, bch);
        const long long nfw = warp_sum((long long)nf);
        if (lane == 0) {
            red[warp] = bc;
            redi[warp] = bch;
        }
        __shared__ long long nfs[kWarps];
        if (lane == 0) nfs[warp] = nfw;
        __syncthreads();
        if (tid == 0) {
            long long b = LLONG_MAX, tot = 0;
            int bi = INT_MAX;
            for (int w = 0; w < kWarps; ++w) {
                tot += nfs[w];
                if (red[w] < b || (red[w] == b && redi[w] < bi)) {
                    b = red[w];
                    bi = redi[w];
                }
            }
            a.feasible_count[j] += tot;
            s_copy = 0;
            if (bi != INT_MAX && b < a.best_cost[j]) {
                a.best_cost[j] = b;
                a.best_iter[j] = (int)iter;
                a.best_chain[j] = bi;
                s_best_chain = bi;
                s_copy = 1;
            }
        }
        __syncthreads();
        if (s_copy)
            for (int w = tid; w < a.words; w += kPostThreads)
                a.best_x[(size_t)j * a.words + w] = a.x[(base + s_best_chain) * a.words + w];
    }

    // Multiplier step (Algorithm 1) with the batch mean of the normalised constraint, under
    // the step-size rule (constant eta and no averaging unless asked).
    if (a.do_lambda && tid < m) {
        const float sg = a.inst[j].sigma_g;
        const double mean = __ddiv_rn((double)gsum[tid], (double)C);
        double eta_k = a.eta;
        if (a.eta_decay != 0.0) {
            double den = __dadd_rn(1.0, __dmul_rn(a.eta_decay, (double)iter));
            if (a.eta_sqrt) den = __dsqrt_rn(den);
            eta_k = __ddiv_rn(a.eta, den);
        }
        double d = mean;
        if (a.momentum != 0.0) {
            double *av = a.avg + (size_t)j * a.m_stride + tid;
            d = __dadd_rn(__dmul_rn(a.momentum, *av), __dmul_rn(__dadd_rn(1.0, -a.momentum), mean));
            *av = d;
        }
        const double step = __dmul_rn(eta_k, __dmul_rn((double)sg, d));
        double l = __dadd_rn((double)a.lambda[(size_t)j * a.m_stride + tid], step);
        if (a.project && l < 0.0) l = 0.0;
        const float nl = __double2float_rn(l);
        a.lambda[(size_t)j * a.m_stride + tid] = nl;
        if (a.lambda_trace)
            a.lambda_trace[((size_t)(iter - a.iter0) * a.count + j) * a.m_stride + tid] = nl;
    }
}

__global__ void advance_iter_kernel(uint32_t *it) { *it += 1u; }

// A device-side check that fails by construction (debug builds): exercises the reporting path.
__global__ void dcheck_selftest_kernel(int32_t *status) {
    const volatile int never = 0;
    (void)SAIS_DCHECK(status, never != 0);
}

}  // namespace

cudaError_t launch_post(const PostArgs &a, cudaStream_t stream) {
    post_kernel<<<a.count, kPostThreads, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_advance_iter(uint32_t *iter_dev, cudaStream_t stream) {
    advance_iter_kernel<<<1, 1, 0, stream>>>(iter_dev);
    return cudaGetLastError();
}

bool debug_checks_built() {
#if defined(SAIS_DEBUG) && SAIS_DEBUG
    return true;
#else
    return false;
#endif
}

cudaError_t launch_dcheck_selftest(int32_t *status, cudaStream_t stream) {
    dcheck_selftest_kernel<<<1, 1, 0, stream>>>(status);
    return cudaGetLastError();
}

}  // namespace sais
