// sais_internal.h -- data shared by the host code and the kernels of libsais.
//
// One instance of the slack-extended, normalised knapsack problem lives on the device as an
// InstDev record plus the arrays it points to.  All arrays of a handle sit in one device pool.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "sais.h"

namespace sais {

// An NVTX range over a scope (entry points, iterations of Algorithm 1): visible in Nsight
// timelines, a few nanoseconds when no tool is attached (NVTX is header-only and loads a tool
// library only if one is injected).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int kMaxConstraints = 32;    // m <= 32: per-chain constraint state lives in registers
constexpr int kMaxBlockedConstraints = 8;   // the blocked sampler keeps 8 at most in registers
constexpr int kSpinPad = 64;           // N' is padded to a multiple of 64 spins
constexpr int kMaxPlainSmem = 220 * 1024;

// Device view of one instance.  Spins are ordered items first, then the slack bits of
// constraint 0, 1, ... (bit q of constraint k has coefficient 2^q in row k of A_ext).
struct InstDev {
    int32_t n;          // items
    int32_t m;          // constraints
    int32_t nprime;     // spins N' = n + sum_k Q_k
    int32_t npad;       // N' rounded up to kSpinPad
    int32_t words;      // ceil(N'/32)
    int32_t has_w;      // 1: quadratic objective (QKP), 0: linear (MKP)
    float sigma_f;      // 1/max(|W|,|h|)
    float sigma_g;      // 1/max(|A|,|b|)
    float P;            // penalty
    float kappa;        // fl(2 P sigma_g^2), FP64 product rounded once
    double psg2;        // P sigma_g^2 in FP64 (exact-path evaluation)
    const int16_t *W;   // npad x npad row-major pair values, zero padded (NULL if !has_w)
    const float *hF;    // npad: h_i as FP32 (exact integers), 0 for slack/padding
    const int32_t *acol;   // npad x m, spin-major: a_ki of A_ext (zero past N')
    const float *acf;      // npad x m4, spin-major: a_ki as FP32 (exact), rows padded to
                           // m4 = m rounded up to 4 with zeros, 16-byte aligned (float4 loads)
    int32_t m4;
    const float *D;        // npad: fl(P sigma_g^2 sum_k a_ki^2) (zero past N')
    const float *asum;     // npad: sum_k a_ki, exact in FP32 (zero past N')
    const float4 *spinc;   // npad: {a_0i, D_i, sum_k a_ki, a_1i}, FP32 (exact integers)
    const int32_t *b;      // m capacities of the sampled problem (B' when tightened)
    const int32_t *fmargin;    // m: a sample is feasible iff g_k - (slack value)_k <= fmargin[k]
                               // (items load <= the caller's capacity; 0 unless tightened)
    const int32_t *slack_off;  // m+1: first slack spin of constraint k; [m] = N'
    // BF16 copy of W for the blocked sampler in its shared-memory image: column-chunk major,
    // element (j, s) at index ((s/8) npad + j) 8 + s%8; Wbf_lo holds W - Wbf when |W| > 256.
    const uint16_t *Wbf;
    const uint16_t *Wbf_lo;
    // The 16 x 16 diagonal blocks of W as FP32 (exact integers), block b at 256 b, row-major:
    // the in-block corrections of the blocked sampler when W is streamed (NULL if !has_w).
    const float *Wdiag;
    // Block-field sampler (sais_field_kernel.cuh).  n16 = n rounded up to 16: the K extent of
    // its GEMM (slack spins have no pair values).  Wg holds W as BF16 with rows in groups of 8:
    // element (i, j), i < npad, j < n16, at index ((i/8)(n16/8) + j/8) 64 + (i%8) 8 + j%8, so the
    // rows of one block of spins form one contiguous K-major MMA operand (core matrices of 8 rows
    // x 8 columns; 128 bytes between column groups, 16 n16 bytes between row groups); Wg_lo is
    // W - Wg when |W| > 256.  Wd32 / Wd64: the 32 x 32 / 64 x 64 diagonal blocks of W in FP32,
    // block b at K^2 b, row-major (K = 16 uses Wdiag).
    int32_t n16;
    const uint16_t *Wg;
    const uint16_t *Wg_lo;
    const float *Wd32;
    const float *Wd64;
};

// Arguments of one sampling launch over all instances of a handle.
struct SampleArgs {
    const InstDev *inst;
    int32_t count;
    int32_t chains;
    int32_t sweeps;
    float beta_max;
    uint32_t iter;
    const uint32_t *iter_dev;  // if not NULL, the outer-iteration index is read here
    uint64_t seed;
    int32_t words;       // stride of x
    int32_t m_stride;    // stride of lambda and g
    const float *lambda;     // [count*m_stride]
    uint32_t *x;             // [count*chains*words]
    int64_t *cost;           // [count*chains]
    int64_t *g;              // [count*chains*m_stride]
    uint8_t *feasible;       // [count*chains] or NULL
    uint32_t *trace;         // [count*chains*sweeps*words] or NULL
    // Best feasible sweep-end state of each run (all NULL: off; run_cost set: on).
    uint32_t *run_x;         // [count*chains*words]
    int64_t *run_cost;       // [count*chains], INT64_MAX when no sweep ended feasible
    int32_t *run_sweep;      // [count*chains] or NULL: the sweep that reached it, -1 if none
    int32_t *run_nfeas;      // [count*chains] or NULL: feasible sweep-end states
    int32_t *status;         // device status word (SAIS_ETIMEOUT etc.), or NULL
    // Ragged launches: work[2 i], work[2 i + 1] = (instance, chain group) of CTA i, nwork
    // entries; NULL = the full grid (chain groups x instances).  inst_chains[j] = chains of
    // instance j (NULL: `chains` for all); `chains` stays the stride of the outputs.
    const int32_t *work;
    int32_t nwork;
    const int32_t *inst_chains;
};

// Arguments of the per-instance post-processing launch (readout reduction, best-so-far,
// multiplier step).
struct PostArgs {
    const InstDev *inst;
    int32_t count;
    int32_t chains;
    int32_t words;
    int32_t m_stride;
    double eta;
    int32_t project;
    double eta_decay;        // step-size rule (0: constant eta)
    int32_t eta_sqrt;        // 1: eta / sqrt(1 + eta_decay k)
    double momentum;         // averaging weight (0: the batch mean)
    double *avg;             // [count*m_stride] running average (momentum != 0)
    int32_t track_best;      // keep the best feasible sample (sais_track_best)
    int32_t do_lambda;       // take the multiplier step (sais_update_lambda)
    const uint32_t *x;
    const int64_t *cost;
    const int64_t *g;
    const uint8_t *feasible;     // NULL: feasible iff cost != INT64_MAX
    float *lambda;           // in/out
    float *lambda_trace;     // [iters*count*m_stride] or NULL
    const uint32_t *iter_dev;    // current iteration (trace row = *iter_dev - iter0)
    uint32_t iter;               // used when iter_dev is NULL
    uint32_t iter0;
    int64_t *best_cost;      // [count]
    uint32_t *best_x;        // [count*words]
    int32_t *best_iter;      // [count]
    int32_t *best_chain;     // [count]
    int64_t *feasible_count; // [count]
    const int32_t *inst_chains;  // chains of instance j (NULL: `chains` for all)
};

// Launchers (defined in the .cu files); they only enqueue work on `stream`.
// f16: F held as int16 in shared memory (every quadratic instance of the launch has
// |h_i| + sum_j |W_ij| <= 32767, so F is exact in it for every state), else FP32.
cudaError_t launch_plain_sampler(const SampleArgs &a, int max_m, int max_npad, int max_words,
                                 int chains_per_cta, cudaStream_t stream, bool f16 = false);
cudaError_t launch_blocked_sampler(const SampleArgs &a, int max_m, int max_npad,
                                   int max_words, int block_k, bool stream_w, bool hilo,
                                   int32_t *status, long long dec_wait_polls,
                                   cudaStream_t stream);
size_t blocked_smem_bytes(int max_npad, int max_words, int block_k, bool stream_w, bool hilo);
// Block-field sampler: each block's fields from one tcgen05 GEMM over the chain states held in
// TMEM and, past 512 columns, in shared memory (W present, m <= 8, n <= 1024).
size_t field_smem_bytes(int max_n16, int max_words, int block_k, bool hilo);
// Accumulator columns of the block-field GEMM: two slots (the GEMM of the next block runs while
// a block is decided) of K columns, or 2K with the hi/lo split (both terms in one MMA of N = 2K).
inline int field_dcols(int block_k, bool hilo) { return 2 * (hilo ? 2 * block_k : block_k); }
uint32_t field_tmem_cols(int max_n16, int dcols);
cudaError_t launch_field_sampler(const SampleArgs &a, int max_m, int max_n16, int max_words,
                                 int block_k, bool hilo, int32_t *status,
                                 long long dec_wait_polls, cudaStream_t stream);
int field_ring(int max_n16, int max_words, int block_k, bool hilo);
int field_xs_chunks(int max_n16, int dcols);
// One persistent launch over a ragged batch's items (instance, chain group, kind): kind 0 / 1
// block-field sampler on 128 chains (m <= 1 / m <= 8), kind 2 / 3 plain sampler on 256 chains
// (m <= 8 / m <= 32); `head` is the device work counter (zeroed by the launch); max_n16_w is the
// largest n16 among the quadratic instances (0 if none).  `stats` receives 4 uint64 per CTA of
// the launch's ragged_grid(nitems, sms) CTAs: start and end on the global timer (ns), time
// inside items (ns) and items run.
constexpr int kRaggedFieldChains = 128, kRaggedPlainItemChains = 256;
size_t ragged_smem_bytes(int max_n16_w, int max_words, bool hilo, int *ring);
int ragged_grid(int nitems, int sms);
cudaError_t launch_ragged(const SampleArgs &a, const int32_t *items, int32_t nitems,
                          int32_t *head, unsigned long long *stats, int max_n16_w,
                          int max_words, bool hilo, int32_t *status, long long dec_wait_polls,
                          int sms, cudaStream_t stream);
size_t plain_smem_bytes(int max_npad, int max_words, bool any_w, int cpb, bool f16 = false);
constexpr size_t kMaxSmemPerBlock = 232448;   // 227 KB opt-in per CTA on sm_103
cudaError_t launch_post(const PostArgs &a, cudaStream_t stream);
cudaError_t launch_advance_iter(uint32_t *iter_dev, cudaStream_t stream);
bool debug_checks_built();   // compiled with SAIS_DEBUG=1
cudaError_t launch_dcheck_selftest(int32_t *status, cudaStream_t stream);

// Device allocations of the library's own buffers: cudaMalloc / cudaFree, or the caller's pair
// installed with sais_set_device_allocator.  dev_alloc returns cudaErrorMemoryAllocation when
// the caller's alloc returns NULL (or memory that is not 256-byte aligned); dev_free releases a
// block with the pair that allocated it (NULL is ignored).
cudaError_t dev_alloc(void **ptr, size_t bytes);
void dev_free(void *ptr);

// Read-only view of a problem handle and access to the sampler dispatch of sais_api.cpp, for
// entry points defined in other translation units.
struct ProblemView {
    int device;
    int count;
    int words;
    int m_stride;
    const InstDev *d_inst;
    int32_t *d_status;
    long long spins_total;   // sum of N' over the instances
    const int32_t *d_inst_chains;   // per-instance chains (device), or NULL
    long long spin_chains_total;    // sum of N' x chains when per-instance chains are set, else 0
};
sais_status problem_view(const sais_problem *p, ProblemView *out);
// run_x / run_cost: best-in-run outputs, or NULL (off).
sais_status enqueue_sample_internal(sais_problem *p, const sais_sample_params *prm,
                                   const float *lambda, const uint32_t *iter_dev, uint32_t *x,
                                   int64_t *cost, int64_t *g, uint8_t *feasible,
                                   uint32_t *run_x, int64_t *run_cost, cudaStream_t stream);
// The argument checks of sais_sample plus every size and variant check of the launch it would
// make (nothing is queued).
sais_status check_sample_params_internal(const sais_problem *p, const sais_sample_params *prm);
// Looks up the device address of sais_solve_noalloc's static scratch on the current device
// (loading the module that holds it, if the CUDA runtime has not yet).  Called when a problem is
// created, so that the first sais_solve_noalloc on that device finds the address ready.
void noalloc_prepare(int device);
sais_status check_step_rule_internal(double eta_decay, double momentum);
sais_status set_error(sais_status s, const char *fmt, ...);
// Inference launch of the warm-start network: lambda[dst[r]] = max(0, y(feat row r)).
sais_status mlp_warm_start_launch(const sais_mlp *m, const float *feat, const int32_t *dst,
                                  int32_t rows, float *lambda, int device, cudaStream_t st);

}  // namespace sais
