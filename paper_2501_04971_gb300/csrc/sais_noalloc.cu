// sais_noalloc.cu -- sais_solve_noalloc: Algorithm 1 without any allocation.
//
// sais_solve allocates device scratch for the samples of each iteration, the kept best sample,
// the multiplier trajectory and an iteration counter.  Some callers cannot allocate device
// memory while they run: code that must not touch the allocator on its hot path (a real-time
// loop, a host that pre-plans every byte of device memory, a plugin handed only its buffers).
// For them this entry point keeps its scratch in one file-scope device array of fixed size,
// kNoAllocScratchBytes, that the GPU holds for as long as the library is loaded.  It calls no
// cudaMalloc, cudaFree, event, graph or other allocating routine, host or device.
//
// Use and limits:
//  * The array's device address is looked up (cudaGetSymbolAddress, with the device current)
//    once per device: when a problem is created on it, or else by the first call.  With the CUDA
//    runtime's lazy module loading, that lookup is what loads this module and so reserves the
//    array; a caller that must not allocate later should create its problems (or make a first
//    call) beforehand, and outside any stream capture.
//  * A call whose scratch would exceed kNoAllocScratchBytes is rejected with SAIS_EINVAL.
//  * All calls share the array.  Calls from this process are serialised by a lock held until the
//    call has synchronised its stream, on every return path once anything has been queued, so two
//    calls never overlap; work that another caller enqueues against the array by other means
//    would race with it.  Every size and variant check runs before anything is queued.
//  * Every region that must start at zero or at a sentinel is set at the start of each call; the
//    rest keeps the previous call's contents and is overwritten before it is read.
#include <chrono>
#include <climits>
#include <cmath>
#include <mutex>

#include "sais_internal.h"

namespace sais {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;   // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_lock;
void *g_scratch_addr[kMaxDevices] = {};

__global__ void init_best_kernel(int64_t *best_cost, int32_t *best_iter, int32_t *best_chain,
                                 int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        best_cost[i] = LLONG_MAX;
        best_iter[i] = -1;
        best_chain[i] = -1;
    }
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Address of the scratch on the current device, looked up once (caller holds the lock).
cudaError_t scratch_address(int device, unsigned char **out) {
    if (!g_scratch_addr[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        if (!ptr) return cudaErrorInvalidSymbol;
        g_scratch_addr[device] = ptr;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[device]);
    return cudaSuccess;
}

}  // namespace

void noalloc_prepare(int device) {
    if (device < 0 || device >= kMaxDevices) return;
    std::lock_guard<std::mutex> lock(g_noalloc_lock);
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    if (cudaSetDevice(device) != cudaSuccess) return;
    unsigned char *ptr = nullptr;
    if (scratch_address(device, &ptr) != cudaSuccess) cudaGetLastError();   // retried at the call
    cudaSetDevice(prev);
}

}  // namespace sais

using namespace sais;

extern "C" sais_status sais_solve_noalloc(sais_problem *p, const sais_solve_params *prm,
                                          sais_solve_result *res, void *stream) {
    if (!p || !prm || !res) return set_error(SAIS_EINVAL, "NULL argument");
    if (prm->iters < 1) return set_error(SAIS_EINVAL, "iters = %d: need >= 1", prm->iters);
    if (!std::isfinite(prm->eta)) return set_error(SAIS_EINVAL, "eta must be finite");
    if (prm->use_graph)
        return set_error(SAIS_EINVAL,
                         "sais_solve_noalloc does not build CUDA graphs (use_graph must be 0)");
    if (prm->variant == SAIS_AUTO)
        return set_error(SAIS_EINVAL,
                         "sais_solve_noalloc takes SAIS_PLAIN or SAIS_BLOCKED (SAIS_AUTO may "
                         "allocate its work list)");
    ProblemView v;
    sais_status st = problem_view(p, &v);
    if (st != SAIS_OK) return st;
    if (v.device < 0 || v.device >= kMaxDevices)
        return set_error(SAIS_EUNSUPPORTED, "device %d beyond the %d supported", v.device,
                         kMaxDevices);
    sais_sample_params sp{};
    sp.chains = prm->chains;
    sp.sweeps = prm->sweeps;
    sp.beta_max = prm->beta_max;
    sp.iter = prm->iter0;
    sp.seed = prm->seed;
    sp.variant = prm->variant;
    sp.block_k = prm->block_k;
    sp.chains_per_cta = prm->chains_per_cta;
    st = check_sample_params_internal(p, &sp);
    if (st != SAIS_OK) return st;
    st = check_step_rule_internal(prm->eta_decay, prm->momentum);
    if (st != SAIS_OK) return st;

    const int count = v.count, C = prm->chains, K = prm->iters;
    const size_t nch = (size_t)count * C;
    const bool rb = prm->run_best != 0;
    const bool avg_on = prm->momentum != 0.0;
    const size_t sizes[15] = {
        (size_t)count * v.m_stride * 4,        // lambda
        nch * v.words * 4,                     // x
        nch * 8,                               // cost
        nch * v.m_stride * 8,                  // g
        nch,                                   // feasible
        (size_t)count * 8,                     // best_cost
        (size_t)count * v.words * 4,           // best_x
        (size_t)count * 4,                     // best_iter
        (size_t)count * 4,                     // best_chain
        (size_t)count * 8,                     // feasible_count
        (size_t)K * count * v.m_stride * 4,    // lambda trace
        4,                                     // iteration counter
        rb ? nch * v.words * 4 : 0,            // best-in-run states
        rb ? nch * 8 : 0,                      // best-in-run costs
        avg_on ? (size_t)count * v.m_stride * 8 : 0};   // averaged subgradients
    size_t offs[15], need = 0;
    for (int i = 0; i < 15; ++i) {
        offs[i] = need;
        need = align256(need + sizes[i]);
    }
    if (need > kNoAllocScratchBytes)
        return set_error(SAIS_EINVAL,
                         "sais_solve_noalloc needs %zu bytes of scratch for %d instances x %d "
                         "chains x %d iterations; its static scratch holds %zu bytes "
                         "(use sais_solve)",
                         need, count, C, K, kNoAllocScratchBytes);

    std::lock_guard<std::mutex> lock(g_noalloc_lock);
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(v.device) != cudaSuccess)
        return set_error(SAIS_ECUDA, "cudaSetDevice(%d) failed", v.device);
    struct Restore {
        int d;
        ~Restore() { cudaSetDevice(d); }
    } restore{prev};
    unsigned char *scr = nullptr;
    {
        cudaError_t e = scratch_address(v.device, &scr);
        if (e != cudaSuccess)
            return set_error(SAIS_ECUDA, "cudaGetSymbolAddress of the static scratch: %s",
                             cudaGetErrorString(e));
    }
    float *d_lam = reinterpret_cast<float *>(scr + offs[0]);
    uint32_t *d_x = reinterpret_cast<uint32_t *>(scr + offs[1]);
    int64_t *d_cost = reinterpret_cast<int64_t *>(scr + offs[2]);
    int64_t *d_g = reinterpret_cast<int64_t *>(scr + offs[3]);
    uint8_t *d_feas = scr + offs[4];
    int64_t *d_bc = reinterpret_cast<int64_t *>(scr + offs[5]);
    uint32_t *d_bx = reinterpret_cast<uint32_t *>(scr + offs[6]);
    int32_t *d_bi = reinterpret_cast<int32_t *>(scr + offs[7]);
    int32_t *d_bch = reinterpret_cast<int32_t *>(scr + offs[8]);
    int64_t *d_fc = reinterpret_cast<int64_t *>(scr + offs[9]);
    float *d_tr = reinterpret_cast<float *>(scr + offs[10]);
    uint32_t *d_iter = reinterpret_cast<uint32_t *>(scr + offs[11]);
    uint32_t *d_rx = rb ? reinterpret_cast<uint32_t *>(scr + offs[12]) : nullptr;
    int64_t *d_rc = rb ? reinterpret_cast<int64_t *>(scr + offs[13]) : nullptr;
    double *d_avg = avg_on ? reinterpret_cast<double *>(scr + offs[14]) : nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Once anything is queued, every return synchronises the stream before the lock is released
    // (this guard is destroyed before `lock`), so a failing call leaves no work on the array.
    struct SyncOnReturn {
        cudaStream_t s;
        bool armed;
        ~SyncOnReturn() {
            if (armed) cudaStreamSynchronize(s);
        }
    } sync_guard{s, false};

#define NOALLOC_CUDA(expr)                                                              \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return set_error(SAIS_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));     \
    } while (0)

    const auto t0 = std::chrono::steady_clock::now();
    sync_guard.armed = true;
    // Regions read before they are written: multipliers, best-so-far state, counters, trace.
    NOALLOC_CUDA(cudaMemsetAsync(d_lam, 0, sizes[0], s));
    NOALLOC_CUDA(cudaMemsetAsync(d_bx, 0, sizes[6], s));
    NOALLOC_CUDA(cudaMemsetAsync(d_fc, 0, sizes[9], s));
    NOALLOC_CUDA(cudaMemsetAsync(d_tr, 0, sizes[10], s));
    if (avg_on) NOALLOC_CUDA(cudaMemsetAsync(d_avg, 0, sizes[14], s));
    if (prm->lambda0)
        NOALLOC_CUDA(cudaMemcpyAsync(d_lam, prm->lambda0, sizes[0], cudaMemcpyHostToDevice, s));
    init_best_kernel<<<(count + 255) / 256, 256, 0, s>>>(d_bc, d_bi, d_bch, count);
    NOALLOC_CUDA(cudaGetLastError());
    NOALLOC_CUDA(cudaMemcpyAsync(d_iter, &prm->iter0, 4, cudaMemcpyHostToDevice, s));

    PostArgs pa{};
    pa.inst = v.d_inst;
    pa.count = count;
    pa.chains = C;
    pa.words = v.words;
    pa.m_stride = v.m_stride;
    pa.eta = prm->eta;
    pa.project = prm->project_nonneg ? 1 : 0;
    pa.eta_decay = prm->eta_decay;
    pa.eta_sqrt = prm->eta_sqrt ? 1 : 0;
    pa.momentum = prm->momentum;
    pa.avg = d_avg;
    pa.track_best = 1;
    pa.do_lambda = 1;
    pa.x = rb ? d_rx : d_x;   // best-in-run: the kept sample of a chain is its best sweep end
    pa.cost = rb ? d_rc : d_cost;
    pa.g = d_g;
    pa.feasible = rb ? nullptr : d_feas;
    pa.lambda = d_lam;
    pa.lambda_trace = d_tr;
    pa.iter_dev = d_iter;
    pa.iter0 = prm->iter0;
    pa.best_cost = d_bc;
    pa.best_x = d_bx;
    pa.best_iter = d_bi;
    pa.best_chain = d_bch;
    pa.feasible_count = d_fc;
    pa.inst_chains = v.d_inst_chains;
    for (int k = 0; k < K; ++k) {
        st = enqueue_sample_internal(p, &sp, d_lam, d_iter, d_x, d_cost, d_g, d_feas, d_rx, d_rc,
                                     s);
        if (st != SAIS_OK) return st;
        NOALLOC_CUDA(launch_post(pa, s));
        NOALLOC_CUDA(launch_advance_iter(d_iter, s));
    }
    if (res->best_cost) NOALLOC_CUDA(cudaMemcpyAsync(res->best_cost, d_bc, sizes[5], cudaMemcpyDeviceToHost, s));
    if (res->best_x) NOALLOC_CUDA(cudaMemcpyAsync(res->best_x, d_bx, sizes[6], cudaMemcpyDeviceToHost, s));
    if (res->best_iter) NOALLOC_CUDA(cudaMemcpyAsync(res->best_iter, d_bi, sizes[7], cudaMemcpyDeviceToHost, s));
    if (res->best_chain) NOALLOC_CUDA(cudaMemcpyAsync(res->best_chain, d_bch, sizes[8], cudaMemcpyDeviceToHost, s));
    if (res->feasible_count) NOALLOC_CUDA(cudaMemcpyAsync(res->feasible_count, d_fc, sizes[9], cudaMemcpyDeviceToHost, s));
    if (res->lambda_final) NOALLOC_CUDA(cudaMemcpyAsync(res->lambda_final, d_lam, sizes[0], cudaMemcpyDeviceToHost, s));
    if (res->lambda_trace) NOALLOC_CUDA(cudaMemcpyAsync(res->lambda_trace, d_tr, sizes[10], cudaMemcpyDeviceToHost, s));
    int32_t status = 0;
    NOALLOC_CUDA(cudaMemcpyAsync(&status, v.d_status, 4, cudaMemcpyDeviceToHost, s));
    NOALLOC_CUDA(cudaStreamSynchronize(s));
    if (status != SAIS_OK) {
        NOALLOC_CUDA(cudaMemsetAsync(v.d_status, 0, 4, s));
        return set_error((sais_status)status, "a sampler kernel reported: %s",
                         sais_status_string((sais_status)status));
    }
    res->elapsed_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    res->spin_updates = (v.spin_chains_total ? (int64_t)v.spin_chains_total
                                              : (int64_t)v.spins_total * C) *
                        (int64_t)prm->sweeps * K;
    return SAIS_OK;
#undef NOALLOC_CUDA
}
