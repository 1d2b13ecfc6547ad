/*
 * sais.h -- C-ABI of libsais, the GB300 (sm_103a) hot path of the Self-Adaptive Ising Machine
 * (SAIM) for constrained binary optimisation: C. Delacour, "Self-Adaptive Ising Machines for
 * Constrained Optimization", arXiv 2501.04971.
 *
 * The method.  A constrained problem  min f(x) s.t. g(x) = 0,  x in {0,1}^N  (Sec. II, Eq. 2)
 * is relaxed into the Lagrange function L = f + P ||g||^2 + lambda^T g (Eq. 3 and 5).  An Ising
 * machine samples low-L states; after each run the multipliers take the subgradient step
 * lambda <- lambda + eta g(x) (Algorithm 1).  The machine is a network of p-bits,
 * I_i = sum_j J_ij m_j + h_i (Eq. 9), m_i = sign(tanh(beta I_i) + rand(-1,1)) (Eq. 10), updated
 * one spin after the other with beta annealed linearly from 0 to beta_max (Sec. III-B).  The
 * problems are knapsacks (Sec. IV): minimise c(x) = -x^T W x / 2 - h^T x subject to A x <= b
 * (QKP: one constraint, W dense; MKP: several constraints, W absent).  Inequalities become
 * equalities with binary slack spins, Q_k = floor(log2 b_k) + 1 per constraint (Sec. IV-A).
 *
 * Conventions used by every entry point.
 *  - Status codes, never exceptions, cross the ABI.  On failure the thread-local message of
 *    sais_last_error() says what was wrong.  No entry point falls back to a CPU path; a device
 *    that is not sm_103 is SAIS_EUNSUPPORTED.
 *  - "host" pointers are ordinary host memory; "device" pointers are CUDA device memory of the
 *    problem's device.  The caller owns every pointer it passes.  sais_create_* copy the problem
 *    data to the device, so host arrays may be freed when they return.  Device buffers passed to
 *    sais_sample / sais_update_lambda are borrowed until the work queued on `stream` completes.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.  All GPU
 *    work of a call is queued on that stream; calls return without synchronising unless stated.
 *  - A problem handle may hold a batch of `count` independent instances.  Per-instance device
 *    arrays are laid out [count][chains][stride], with strides given by sais_problem_info:
 *    words = ceil(max N'/32) for bit-packed states (spin i of a chain is bit i%32 of word i/32),
 *    m_stride = max(1, max m) for per-constraint values.  Unused tail entries are written 0.
 *  - Spin order: items 0..n-1, then the slack bits of constraint 0 (bit q has coefficient 2^q),
 *    then those of constraint 1, and so on.
 *  - Random numbers: instance j of a batch draws from Philox4x32-10 with key (seed + j, as two
 *    32-bit words, low first) and counter (i/4, sweep t, chain c, outer iteration k); word i%4
 *    gives rho = (2v+1)/2^24 - 1, v = word >> 8.  Equal arguments give equal results on every run.
 *  - Scalars (sigma_f, sigma_g, P, beta_t, lambda) are FP32 values; the decision of Eq. 10 is the
 *    one exact real arithmetic on those values gives, evaluated in FP32 with a rigorous error
 *    bound and re-evaluated in FP64 when the bound cannot separate the two outcomes.
 */
#ifndef SAIS_H
#define SAIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SAIS_API __attribute__((visibility("default")))
#else
#define SAIS_API
#endif

typedef enum sais_status {
    SAIS_OK = 0,
    SAIS_EINVAL = 1,       /* bad argument: NULL where data is required, size out of range,
                              W not symmetric / nonzero diagonal, b <= 0, A < 0, ...        */
    SAIS_ENOMEM = 2,       /* a device or host allocation failed                             */
    SAIS_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed                    */
    SAIS_EOVERFLOW = 4,    /* an integer bound that keeps the fields exact would be broken:
                              |h_i| + sum_j |W_ij| >= 2^24, |W_ij| > 32767, or
                              b_k + sum_i a_ki(ext) >= 2^24                                 */
    SAIS_ETIMEOUT = 5,     /* a bounded device wait gave up (status word set by a kernel)    */
    SAIS_EUNSUPPORTED = 6, /* device is not sm_103, or sizes exceed what a kernel supports   */
    SAIS_EBOUNDS = 7       /* debug builds only (compiled with SAIS_DEBUG=1): a device-side
                              check of an index or size failed; the kernel skipped the access
                              and its outputs are not valid (sais_last_error names the check's
                              source line)                                                  */
} sais_status;

/* One knapsack instance in integer form (Sec. IV, Eq. 12 and 14):
 *   minimise  c(x) = -x^T W x / 2 - h^T x   subject to   A x <= b,   x in {0,1}^n.
 * All arrays are host memory, read during sais_create_* only. */
typedef struct sais_problem_desc {
    int32_t n;          /* items, >= 1                                                      */
    int32_t m;          /* constraints (knapsacks), 0 <= m <= 32                            */
    const int32_t *W;   /* n*n row-major pair values, symmetric, zero diagonal, |W_ij| <=
                           32767; NULL for a linear objective (MKP)                          */
    const int32_t *h;   /* n item values                                                    */
    const int32_t *A;   /* m*n row-major weights, >= 0 (may be NULL when m == 0)            */
    const int64_t *b;   /* m capacities, >= 1                                               */
    float alpha;        /* penalty rule P = alpha d N' (Sec. III-A; Table I: QKP 2, MKP 5)  */
    float density;      /* d in the penalty rule; < 0 selects the measured profit density
                           (QKP: nonzero p_ij, i <= j, over n(n+1)/2) or 2/(N'+1) when W is
                           NULL (Sec. IV-B)                                                   */
    float penalty;      /* > 0: use this P instead of the alpha rule                        */
    const int64_t *b_tight; /* NULL, or m reduced capacities B'_k, 1 <= B'_k <= b_k: capacity
                           tightening (Sec. IV-B).  The sampled problem is the one with
                           capacities B' in full (slack bits, sigma_g, g, penalty rule); the
                           feasibility test and the kept best samples use b.  A zero-
                           initialised descriptor leaves it NULL.                            */
} sais_problem_desc;

/* Scalars derived from one instance on the host (no GPU involved). */
typedef struct sais_problem_scalars {
    int32_t n, m;
    int32_t n_spins;         /* N' = n + sum_k Q_k                                          */
    int32_t words;           /* ceil(N'/32)                                                 */
    float sigma_f;           /* 1 / max(|W|, |h|)            (Sec. IV-A)                    */
    float sigma_g;           /* 1 / max(|A|, |b|)            (Sec. IV-A)                    */
    float penalty;           /* P                             (Sec. III-A)                  */
    float reserved;
    double density;          /* the d that entered P                                        */
} sais_problem_scalars;

typedef struct sais_problem sais_problem; /* opaque, owned by the library */

typedef struct sais_layout {
    int32_t count;           /* instances in the handle                                     */
    int32_t max_spins;       /* max N' over the instances                                   */
    int32_t words;           /* ceil(max N' / 32): stride of bit-packed states              */
    int32_t m_stride;        /* max(1, max m): stride of per-constraint arrays              */
    int32_t device;          /* CUDA device ordinal                                         */
    int32_t has_quadratic;   /* 1 if any instance has W                                     */
} sais_layout;

/* SAIS_PLAIN and SAIS_BLOCKED take at most 65535 instances per handle (one grid row each);
 * SAIS_AUTO takes any number. */
typedef enum sais_variant {
    SAIS_PLAIN = 0,          /* per-spin sampler: FP32 fields, rank-1 update on every flip  */
    SAIS_BLOCKED = 1,        /* k spins per block, field updates on the tensor cores        */
    SAIS_AUTO = 2            /* ragged batches: by default one persistent launch whose CTAs
                                take (instance, chain group) items, most expensive first,
                                from a device counter: the blocked sampler (block fields by
                                GEMM, K = 16) for quadratic objectives with m <= 8 and
                                n <= 1024, the plain sampler for linear ones with m <= 32.
                                Batches outside that (or when sais_autotune measured them
                                faster) run as concurrent launch groups: per group the
                                blocked sampler where an instance allows it, the plain one
                                otherwise, or sais_autotune's choices                       */
} sais_variant;

/* What sais_autotune chose for each launch group of SAIS_AUTO (first 16 groups). */
typedef struct sais_tuning {
    int32_t groups;                  /* launch groups of the batch                         */
    int32_t blocked_instances;       /* instances now run by the blocked sampler           */
    int32_t plain_instances;         /* instances now run by the plain sampler             */
    int32_t reserved;
    int32_t group_variant[16];       /* sais_variant chosen per group                      */
    int32_t group_block_k[16];       /* block size (blocked groups)                        */
    int32_t group_chains_per_cta[16];/* chains per CTA                                     */
    int32_t group_size[16];          /* instances per group                                */
    double group_ms[16];             /* measured time of the chosen configuration          */
    int64_t group_spin_updates[16];  /* spin updates of one timed launch of the group      */
    int32_t persistent_ok;           /* 1: the batch fits one persistent launch            */
    int32_t persistent;              /* 1: SAIS_AUTO now runs the persistent launch, 0: the
                                        group launches (the faster of the two timings)     */
    double persistent_ms;            /* one timed SAIS_AUTO launch, persistent (0 if n/a)  */
    double groups_ms;                /* the same with the concurrent group launches        */
} sais_tuning;

/* One annealing run per chain (Sec. III-B): every chain starts at x = 0 and performs `sweeps`
 * sequential sweeps, sweep t at beta_t = beta_max t / (sweeps-1) (beta_max when sweeps = 1). */
typedef struct sais_sample_params {
    int32_t chains;          /* chains per instance, >= 1                                   */
    int32_t sweeps;          /* T >= 1                                                      */
    float beta_max;          /* >= 0                                                        */
    uint32_t iter;           /* outer-iteration index k (selects the random stream)         */
    uint64_t seed;           /* instance j uses seed + j                                    */
    int32_t variant;         /* sais_variant                                                */
    int32_t block_k;         /* SAIS_BLOCKED: spins per block (16 or 32); 0 = default (16)   */
    int32_t chains_per_cta;  /* 0 = library choice; else 32, 64 or 128                      */
    int32_t debug_wait_polls; /* 0 = normal.  > 0 (fault-injection tests of the timeout path):
                                the blocked sampler's decision warps first wait, for at most
                                this many polls, on a barrier nothing completes, so the kernel
                                stops early, records SAIS_ETIMEOUT (see sais_synchronize),
                                releases its resources and exits; outputs are not written   */
} sais_sample_params;

/* Algorithm 1 (Sec. III-A) on every instance of the handle. */
typedef struct sais_solve_params {
    int32_t iters;           /* K outer iterations, >= 1                                    */
    int32_t chains;          /* chains per instance per iteration (the batch of samples)    */
    int32_t sweeps;          /* sweeps per annealing run                                    */
    float beta_max;
    double eta;              /* step size of the multiplier update                          */
    uint64_t seed;
    uint32_t iter0;          /* index of the first iteration (resume: previous iter0 + K)   */
    int32_t project_nonneg;  /* 1: lambda <- max(0, .) after each step                      */
    int32_t variant;         /* sais_variant of the sampler                                 */
    int32_t block_k;         /* as in sais_sample_params                                    */
    int32_t chains_per_cta;  /* as in sais_sample_params                                    */
    int32_t use_graph;       /* 1: replay the iteration as a captured CUDA graph            */
    const float *lambda0;    /* host [count*m_stride] initial multipliers, or NULL for 0    */
    int32_t run_best;        /* 1: the sample kept from each chain is its best feasible
                                sweep-end state (sais_sample_run_best) instead of its last
                                state; the multipliers still step on the last states        */
    double eta_decay;        /* step-size rule of sais_update_lambda_rule (0: constant eta) */
    int32_t eta_sqrt;        /* 1: eta / sqrt(1 + eta_decay k) instead of eta / (1 + ...)   */
    double momentum;         /* averaging weight mu in [0, 1) (0: the batch mean itself); the
                                average starts at 0 in every call                           */
} sais_solve_params;

/* Results of sais_solve, all caller-allocated HOST arrays (any may be NULL to skip it). */
typedef struct sais_solve_result {
    int64_t *best_cost;      /* [count] min c(x) over the stored feasible samples (Alg. 1,
                                final line); INT64_MAX when none was feasible               */
    uint32_t *best_x;        /* [count*words] the sample achieving it (first in (k, chain)
                                order on ties)                                              */
    int32_t *best_iter;      /* [count] its outer iteration k, -1 if none                   */
    int32_t *best_chain;     /* [count] its chain, -1 if none                               */
    int64_t *feasible_count; /* [count] feasible samples seen                               */
    float *lambda_final;     /* [count*m_stride] multipliers after the last step            */
    float *lambda_trace;     /* [iters*count*m_stride] multipliers after each step          */
    double elapsed_ms;       /* sais_solve: device time of the iterations (CUDA events);
                                sais_solve_noalloc: host wall time of the whole call (its
                                copies and the final synchronisation included), so the two
                                are not like for like                                        */
    int64_t spin_updates;    /* count * chains * sweeps * N' summed over instances and k    */
} sais_solve_result;

/* Slack extension, normalisation and penalty of one instance, computed on the host
 * (Sec. III-A, IV-A, IV-B).  No GPU is touched.  Errors: SAIS_EINVAL, SAIS_EOVERFLOW. */
SAIS_API sais_status sais_describe(const sais_problem_desc *desc, sais_problem_scalars *out);

/* Validate one instance, build its slack-extended, normalised device form on `device` and
 * return a handle in *out.  Errors: SAIS_EINVAL, SAIS_EOVERFLOW, SAIS_ENOMEM, SAIS_ECUDA,
 * SAIS_EUNSUPPORTED (device not sm_103, or N' beyond the kernels' limit). */
SAIS_API sais_status sais_create_problem(const sais_problem_desc *desc, int32_t device,
                                         sais_problem **out);

/* As sais_create_problem for `count` independent instances (descs[0..count-1]) held by one
 * handle; instances may differ in n, m and N'. */
SAIS_API sais_status sais_create_batch(const sais_problem_desc *descs, int32_t count,
                                       int32_t device, sais_problem **out);

/* Free the device data of a handle (synchronises its device).  NULL is accepted. */
SAIS_API sais_status sais_destroy_problem(sais_problem *p);

SAIS_API sais_status sais_problem_info(const sais_problem *p, sais_layout *out);

/* Scalars of instance `index` of a handle (as sais_describe computed them at creation). */
SAIS_API sais_status sais_instance_scalars(const sais_problem *p, int32_t index,
                                           sais_problem_scalars *out);

/* The Ising-machine step of Algorithm 1 ("minimise L_k") as Sec. III-B runs it: one annealing
 * run of p-bit Gibbs sweeps per chain at multipliers `lambda`, returning each chain's last
 * sample x_k with its cost and constraint values.
 *   lambda   device [count*m_stride] FP32 multipliers (read)
 *   x        device [count*chains*words] bit-packed last samples (written)
 *   cost     device [count*chains] int64 c(x) = -x^T W x / 2 - h^T x (written)
 *   g        device [count*chains*m_stride] int64 g_k(x) = A_ext x - b, slack included
 *   feasible device [count*chains] uint8, 1 iff A x <= b on the items (Sec. IV-A), or NULL
 *            (b: the descriptor's capacities, also when b_tight is set)
 * Errors: SAIS_EINVAL (NULL buffers, chains < 1, sweeps < 1, beta_max < 0 or not finite, bad
 * block_k / chains_per_cta), SAIS_EUNSUPPORTED, SAIS_ECUDA (launch failure). */
SAIS_API sais_status sais_sample(sais_problem *p, const sais_sample_params *prm,
                                 const float *lambda, uint32_t *x, int64_t *cost, int64_t *g,
                                 uint8_t *feasible, void *stream);

/* sais_sample that also records the state after every sweep:
 *   trace  device [count*chains*sweeps*words] bit-packed states (written)
 * Used to replay recorded sweeps decision by decision against a reference. */
SAIS_API sais_status sais_sample_trace(sais_problem *p, const sais_sample_params *prm,
                                       const float *lambda, uint32_t *x, int64_t *cost,
                                       int64_t *g, uint8_t *feasible, uint32_t *trace,
                                       void *stream);

/* sais_sample that also keeps, per chain, the best feasible state among the states at the ends
 * of the sweeps of its run.  The paper measures one sample per run, its last state (Sec. IV-A);
 * this option measures every sweep end, so a feasible state passed mid-run is not lost (the
 * oracle's run-best option).  x, cost, g and feasible are the last samples as in sais_sample
 * (the multiplier step uses them); in addition:
 *   run_x      device [count*chains*words] the least-cost sweep-end state that is feasible
 *              (A x <= b on the items), the earliest sweep on ties; zeros if none (written)
 *   run_cost   device [count*chains] int64 its cost c(x), INT64_MAX if none (written)
 *   run_sweep  device [count*chains] int32 its sweep t, -1 if none, or NULL
 *   run_nfeas  device [count*chains] int32 number of feasible sweep-end states, or NULL
 * sais_track_best takes run_x and run_cost (with feasible = NULL) to keep the best of a solve.
 * Errors: as sais_sample. */
SAIS_API sais_status sais_sample_run_best(sais_problem *p, const sais_sample_params *prm,
                                          const float *lambda, uint32_t *x, int64_t *cost,
                                          int64_t *g, uint8_t *feasible, uint32_t *run_x,
                                          int64_t *run_cost, int32_t *run_sweep,
                                          int32_t *run_nfeas, void *stream);

/* The multiplier step of Algorithm 1, lambda_k <- lambda_k + eta g_k(x), with the normalised
 * constraint sigma_g g averaged over the `chains` samples of each instance and, if
 * project_nonneg, projected on lambda >= 0.  The chain sum is exact (int64); mean and step are
 * FP64 evaluated as mean = S/C, step = eta*(sigma_g*mean), lambda + step, rounded to FP32.
 *   g       device [count*chains*m_stride] int64 (read), as written by sais_sample
 *   lambda  device [count*m_stride] FP32 (read and written in place)
 * Errors: SAIS_EINVAL, SAIS_ECUDA. */
SAIS_API sais_status sais_update_lambda(sais_problem *p, const int64_t *g, int32_t chains,
                                        double eta, int32_t project_nonneg, float *lambda,
                                        void *stream);

/* sais_update_lambda with a step-size rule (not in the paper).  Sec. III-A relies on the
 * surrogate-gradient method, which lets the step shrink and the direction combine recent
 * subgradients.  With k = iter (the outer-iteration index) and per constraint:
 *   eta_k = eta / (1 + eta_decay k), or eta / sqrt(1 + eta_decay k) when eta_sqrt = 1;
 *   d = momentum avg + (1 - momentum) mean  (avg: the running average, written back);
 *   lambda <- lambda + eta_k (sigma_g d), projected on lambda >= 0 if project_nonneg.
 * FP64 in that order (mean = S/C; den = 1 + eta_decay*k, its square root if asked;
 * eta_k = eta/den, or eta when eta_decay = 0), each operation rounded once, lambda stored as
 * FP32.  eta_decay = 0 and momentum = 0 give sais_update_lambda bit for bit.
 *   avg     device [count*m_stride] FP64 (read and written; start at 0), or NULL when
 *           momentum = 0
 * Errors: SAIS_EINVAL (eta_decay < 0 or not finite, momentum outside [0, 1), avg NULL with
 * momentum != 0), SAIS_ECUDA. */
SAIS_API sais_status sais_update_lambda_rule(sais_problem *p, const int64_t *g, int32_t chains,
                                             double eta, int32_t project_nonneg, uint32_t iter,
                                             double eta_decay, int32_t eta_sqrt,
                                             double momentum, double *avg, float *lambda,
                                             void *stream);

/* The "store feasible x_k" step of Algorithm 1 for one batch of samples (Sec. III-A; the
 * feasibility test of Sec. IV-A): among the chains whose sample is feasible, the one of least
 * cost (lowest chain index on ties) replaces the kept best of its instance when it is strictly
 * better, so the kept sample is the first achiever in (iteration, chain) order; the number of
 * feasible samples is added to feasible_count.
 *   x, cost, feasible   device, as written by sais_sample for `chains` chains (read);
 *                       feasible may be NULL: then a sample is feasible iff its cost is not
 *                       INT64_MAX (the run_x / run_cost outputs of sais_sample_run_best)
 *   iter                outer iteration of the samples (stored with a new best)
 *   best_cost       device [count] int64 (in/out; start at INT64_MAX)
 *   best_x          device [count*words] (in/out)
 *   best_iter, best_chain  device [count] int32 (in/out; start at -1)
 *   feasible_count  device [count] int64 (in/out; start at 0)
 * Errors: SAIS_EINVAL, SAIS_ECUDA. */
SAIS_API sais_status sais_track_best(sais_problem *p, const uint32_t *x, const int64_t *cost,
                                     const uint8_t *feasible, int32_t chains, uint32_t iter,
                                     int64_t *best_cost, uint32_t *best_x, int32_t *best_iter,
                                     int32_t *best_chain, int64_t *feasible_count,
                                     void *stream);

/* Algorithm 1 for `iters` iterations on every instance: per iteration one sais_sample batch,
 * the feasible samples checked and the best kept, then sais_update_lambda.  The library owns
 * the device scratch it needs for the call.  Synchronises `stream` before returning and fills
 * the host arrays of `res`.  Errors: as sais_sample, plus SAIS_ENOMEM. */
SAIS_API sais_status sais_solve(sais_problem *p, const sais_solve_params *prm,
                                sais_solve_result *res, void *stream);

/* sais_solve without any allocation.  The paper has no counterpart: this is a deployment
 * variant for callers that cannot allocate memory while they run (a real-time or latency-
 * critical loop that must not enter the allocator, a host that plans every byte of device memory
 * up front, a plug-in handed only its own buffers).  Same parameters and results as sais_solve
 * (use_graph must be 0, variant SAIS_PLAIN or SAIS_BLOCKED: SAIS_AUTO may allocate its work
 * list); the device scratch lives in one static array of 16 MiB that every GPU
 * loading the library holds until the process exits, and the call makes no cudaMalloc, cudaFree,
 * event or graph call, host or device.
 *  - The array's device address is looked up once per device, when a problem is created on it
 *    (or else by the first call).  The CUDA runtime loads modules lazily by default, and this
 *    lookup loads the library's module holding the array, so that is when the 16 MiB are
 *    reserved: a caller that must not allocate later creates its problems beforehand, outside
 *    any stream capture.
 *  - Sizes whose scratch would exceed 16 MiB are rejected with SAIS_EINVAL (the message gives the
 *    bytes needed); sais_solve has no such limit.
 *  - Calls share the array; calls from one process are serialised by a lock held until the
 *    call's stream has synchronised (on every return, once anything has been queued; every size
 *    and variant check runs before that), and calls that overlapped on the GPU by other means
 *    would race.  Regions that must start at zero or at a sentinel are reset by every call.
 * Synchronises `stream` before returning; elapsed_ms is host wall time of the call.
 * Errors: as sais_solve. */
SAIS_API sais_status sais_solve_noalloc(sais_problem *p, const sais_solve_params *prm,
                                        sais_solve_result *res, void *stream);

/* Ragged batches: counts[j] >= 1 chains for instance j (host array of `count` entries, copied);
 * NULL restores one count for all.  While set, the `chains` argument of sais_sample,
 * sais_update_lambda, sais_track_best and sais_solve is the row stride of per-chain arrays
 * (>= every counts[j]); instance j uses its first counts[j] rows, and the multiplier step
 * averages over them.  Errors: SAIS_EINVAL, SAIS_ENOMEM, SAIS_ECUDA. */
SAIS_API sais_status sais_set_instance_chains(sais_problem *p, const int32_t *counts);

/* Autotuner of SAIS_AUTO: for every launch group, times one launch of `sweeps` sweeps with
 * `chains` chains for each candidate (blocked with block_k 16 / 32 / 64 where W allows it,
 * plain with 32 / 64 / 128 chains per CTA) and keeps the fastest; then times one SAIS_AUTO
 * launch as concurrent group launches and one as the persistent launch (when the batch fits
 * it) and keeps the faster mode for later SAIS_AUTO launches.  Allocates and frees temporary
 * device buffers; synchronises `stream`.  Errors: SAIS_EINVAL, SAIS_ENOMEM, SAIS_ECUDA. */
SAIS_API sais_status sais_autotune(sais_problem *p, int32_t chains, int32_t sweeps,
                                   sais_tuning *out, void *stream);

/* The launch sais_sample would make for these parameters, decided from the handle alone
 * (no GPU work): which sampler kernel, its block size and CTA shape.  Errors: those
 * sais_sample reports before launching (SAIS_EINVAL, SAIS_EUNSUPPORTED).  No counterpart in the
 * paper: introspection of the samplers of Sec. III-B as this library runs them. */
typedef enum sais_kernel {
    SAIS_KERNEL_PLAIN = 0,          /* per-spin sampler                                       */
    SAIS_KERNEL_RANKK_RESIDENT = 1, /* blocked, rank-k field update, W resident in SMEM       */
    SAIS_KERNEL_RANKK_STREAMED = 2, /* blocked, rank-k field update, W tiles streamed          */
    SAIS_KERNEL_BLOCK_FIELD = 3,    /* blocked, each block's fields from a GEMM over the states */
    SAIS_KERNEL_GROUPS = 4,         /* SAIS_AUTO: one launch per group (see sais_autotune)     */
    SAIS_KERNEL_PERSISTENT = 5      /* SAIS_AUTO: one persistent launch over the batch's items  */
} sais_kernel;

typedef struct sais_plan {
    int32_t kernel;          /* sais_kernel                                                  */
    int32_t block_k;         /* spins per block (blocked kernels), else 0                    */
    int32_t chains_per_cta;  /* chains per CTA (0 for SAIS_AUTO)                              */
    int32_t hilo;            /* 1 when W is applied as two BF16 terms (pair values > 256)    */
} sais_plan;

SAIS_API sais_status sais_sample_plan(const sais_problem *p, const sais_sample_params *prm,
                                      sais_plan *out);

/* How SAIS_AUTO runs this handle's batch from now on: SAIS_AUTO_PERSISTENT (the default) makes
 * one persistent launch when the batch fits it (see sais_variant) and the group launches
 * otherwise; SAIS_AUTO_GROUPS always makes the group launches.  Both draw identical samples.
 * Overrides the mode sais_autotune chose (and a later sais_autotune overrides this).  No
 * counterpart in the paper: a launch-shape choice for the batched sampler of Sec. III-B.
 * Errors: SAIS_EINVAL (NULL handle or unknown mode). */
typedef enum sais_auto_mode {
    SAIS_AUTO_PERSISTENT = 0,
    SAIS_AUTO_GROUPS = 1
} sais_auto_mode;

SAIS_API sais_status sais_set_auto_mode(sais_problem *p, int32_t mode);

/* Per-CTA record of the most recent persistent launch of this handle (one CTA per SM, at most
 * one per item): waits for `stream`, then copies 4 uint64 per CTA into `out` (host, room for
 * `cap` CTAs): start and end of the CTA on the GPU's global timer (ns), the time it spent
 * running items (ns), and the number of items it ran.  *ctas receives the launch's CTA count
 * (records beyond `cap` are not copied).  Before any persistent launch the records are zero.
 * No counterpart in the paper: load-balance instrumentation of the batched sampler.
 * Errors: SAIS_EINVAL (NULL argument, or no persistent launch prepared for this handle),
 * SAIS_ECUDA. */
SAIS_API sais_status sais_persistent_stats(sais_problem *p, uint64_t *out, int32_t cap,
                                           int32_t *ctas, void *stream);

/* Wait for the work queued on `stream` and report device-side failures of this problem's
 * kernels since the last call: SAIS_ETIMEOUT if a bounded wait inside a kernel gave up (the
 * kernel then stopped early and its outputs are not valid).  Resets the device status word.
 * Errors: SAIS_EINVAL, SAIS_ECUDA, SAIS_ETIMEOUT. */
SAIS_API sais_status sais_synchronize(sais_problem *p, void *stream);

/* Debug builds (SAIS_DEBUG=1): queues on `stream` one kernel whose device-side check fails by
 * construction, so that the next sais_synchronize reports SAIS_EBOUNDS with that check's line
 * (a test of the reporting path; the kernel touches no memory but the status words).  Release
 * builds return SAIS_EUNSUPPORTED and queue nothing.  No counterpart in the paper.
 * Errors: SAIS_EINVAL, SAIS_ECUDA, SAIS_EUNSUPPORTED. */
SAIS_API sais_status sais_debug_check_selftest(sais_problem *p, void *stream);

/* ---- Learned multiplier warm start (the paper has no counterpart) -------------------------
 * A 7 -> 128 -> 128 -> 1 ReLU network (BF16 weights, FP32 accumulation, tensor cores) maps the
 * features of one constraint k of an instance to the multiplier lambda_k that Algorithm 1
 * (Sec. III-A) converges to, so that a run can start from it instead of lambda = 0.
 *
 * Features (8 floats per constraint, column 7 unused), from Sec. IV-A's normalised data:
 *   f0 = min(1, b_k / sum_i a_ki) (1 if the row sum is 0); f1, f2 = sigma_g x mean, population
 *   std of a_ki over the items; f3, f4 = sigma_f x mean, std of the nonzero profits h_i and
 *   W_ij (i < j); f5 = n / 1000; f6 = d, the density that entered P = alpha d N'.
 * Parameters: SAIS_MLP_PARAMS floats, W1 [128 x 16] at 0 (column 7 = b1, columns 8..15 zero),
 *   W2 [128 x 144] at 2048 (column 128 = b2, columns 129..143 zero), w3 [128] at 20480, b3 at
 *   20608, three unused.  Normalisation norm[16] = {mu[7], sd[7], y_mu, y_sd}: the network sees
 *   (f - mu) / sd and predicts lambda = y_mu + y_sd u.
 * The handle owns its device buffers (FP32 master weights, Adam moments, BF16 images of the
 * weights, partial gradients); one stream at a time per handle. */
#define SAIS_MLP_PARAMS 20612
#define SAIS_MLP_FEATURES 8
typedef struct sais_mlp sais_mlp;

/* Features of every constraint of every instance, rows in instance order then k (host array
 * of capacity_rows x 8 floats; *rows receives sum_j m_j).  Errors: SAIS_EINVAL when NULL or
 * the capacity is short. */
SAIS_API sais_status sais_constraint_features(const sais_problem *p, float *out,
                                              int32_t capacity_rows, int32_t *rows);

/* New network on `device`, weights drawn from `seed` (He-uniform hidden layers, zero biases),
 * identity normalisation.  Errors: SAIS_EINVAL, SAIS_ENOMEM, SAIS_ECUDA. */
SAIS_API sais_status sais_mlp_create(int32_t device, uint64_t seed, sais_mlp **out);
SAIS_API sais_status sais_mlp_destroy(sais_mlp *m);

/* Host copies in and out of the parameter vector and (if not NULL) the normalisation.
 * set_params zeroes the padding entries, resets Adam and synchronises the device. */
SAIS_API sais_status sais_mlp_set_params(sais_mlp *m, const float *params, const float *norm);
SAIS_API sais_status sais_mlp_get_params(const sais_mlp *m, float *params, float *norm);

/* Normalisation from a training set on the host: per-feature mean and population std of X
 * (rows x 8) and of the targets y (std < 1e-6 is replaced by 1). */
SAIS_API sais_status sais_mlp_fit_normalization(sais_mlp *m, const float *X, const float *y,
                                                int32_t rows);

/* lambda predicted for each row of X (device, rows x 8) into y (device, rows), not clamped. */
SAIS_API sais_status sais_mlp_forward(const sais_mlp *m, const float *X, int32_t rows, float *y,
                                      void *stream);

/* Gradient of the mean squared error (1/rows) sum (u - t')^2 on normalised targets
 * t' = (t - y_mu) / y_sd, into grad (device, SAIS_MLP_PARAMS floats), and the loss into *loss
 * (device, may be NULL).  X, t on the device. */
SAIS_API sais_status sais_mlp_gradient(sais_mlp *m, const float *X, const float *t, int32_t rows,
                                       float *grad, float *loss, void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8 as FP32 values; bias corrections from those
 * values) of that loss over all `rows` rows. */
SAIS_API sais_status sais_mlp_train_step(sais_mlp *m, const float *X, const float *t,
                                         int32_t rows, float lr, float *loss, void *stream);

/* Device-side failures of the handle's kernels since the last call (SAIS_ETIMEOUT if a bounded
 * wait gave up); resets the status word.  Synchronises the device. */
SAIS_API sais_status sais_mlp_status(sais_mlp *m);

/* Warm start: lambda[j m_stride + k] = max(0, network(features of constraint k of instance j))
 * for every k < m_j (device array of count x m_stride floats; other entries untouched).
 * Errors: SAIS_EINVAL (NULL, other device), SAIS_ECUDA. */
SAIS_API sais_status sais_warm_start(sais_problem *p, const sais_mlp *m, float *lambda,
                                     void *stream);

/* ---- Device memory of the library's own buffers -------------------------------------------
 * The library allocates device memory for problem data (sais_create_*), the per-call scratch of
 * sais_solve and sais_autotune, SAIS_AUTO work lists, per-instance chain counts and the
 * warm-start network's buffers.  By default these come from cudaMalloc / cudaFree.  A caller
 * that manages device memory itself (a memory pool, a framework's caching allocator, a budget
 * that must account for every byte) installs its own pair here; the paper has no counterpart.
 *   alloc(bytes, device, ctx) returns device memory of `device` (the current device when it is
 *     called), at least 256-byte aligned, or NULL on failure (the calling entry point then
 *     returns SAIS_ENOMEM);
 *   free(ptr, bytes, device, ctx) releases a block alloc returned.
 * Process-wide; both NULL restores cudaMalloc / cudaFree.  Every block is freed with the pair
 * that allocated it, whatever is installed by then.  The functions may be called from any
 * thread that calls the library, and must not call back into it.  sais_solve_noalloc makes no
 * allocation either way.  Errors: SAIS_EINVAL when exactly one of the two is NULL. */
typedef void *(*sais_device_alloc_fn)(size_t bytes, int32_t device, void *ctx);
typedef void (*sais_device_free_fn)(void *ptr, size_t bytes, int32_t device, void *ctx);
SAIS_API sais_status sais_set_device_allocator(sais_device_alloc_fn alloc_fn,
                                               sais_device_free_fn free_fn, void *ctx);

/* Static text for a status code. */
SAIS_API const char *sais_status_string(sais_status s);

/* Message of the last failing call on this thread ("" if none). */
SAIS_API const char *sais_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SAIS_H */
