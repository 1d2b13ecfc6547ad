// sais_api.cpp -- host side of libsais: argument checks, the slack-extended and normalised
// device form of each instance, and the entry points declared in include/sais.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "sais.h"
#include "sais_internal.h"

using namespace sais;

namespace {

thread_local std::string g_last_error;

sais_status fail(sais_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

#define SAIS_CUDA(expr)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? SAIS_ENOMEM : SAIS_ECUDA,      \
                        "%s: %s", #expr, cudaGetErrorString(e_));                         \
    } while (0)

constexpr int64_t kExact24 = int64_t(1) << 24;

int32_t binary_digits(int64_t b) {  // Q = floor(log2 b) + 1 for b >= 1 (Sec. IV-A)
    int32_t q = 0;
    for (; b > 0; b >>= 1) ++q;
    return q;
}

// One instance after validation, slack extension and normalisation (host copy).
struct HostInst {
    int32_t n = 0, m = 0, nprime = 0, npad = 0, words = 0;
    bool has_w = false;
    float sf = 1.f, sg = 1.f, P = 0.f;
    double d = 0.0, psg2 = 0.0;
    float kappa = 0.f;
    bool need_lo = false;                  // lo image allocated (BF16 hi/lo split)
    bool lo_own = false;                   // this instance has |W| > 256
    bool f16 = false;                      // every |h_i| + sum_j |W_ij| <= 32767: the plain
                                           // sampler may hold F as int16 (exact)
    std::vector<int32_t> Q, slack_off;     // m, m+1
    std::vector<int32_t> acol;             // nprime x m (spin-major)
    std::vector<float> D, asum;            // npad
    std::vector<float> spinc;              // npad x 4: a_0, D, sum a, a_1 (FP32, exact)
    std::vector<int32_t> b;                // m capacities of the sampled problem (B' if tightened)
    std::vector<int32_t> margin;           // m: b_k - B'_k capped at sum_i a_ki (0 untightened)
    std::vector<float> hF;                 // npad
    std::vector<float> feat;               // m x 8 features of the warm-start network
    const int32_t *W = nullptr;            // borrowed from the descriptor during creation
};

sais_status build_host(const sais_problem_desc *d, HostInst &h) {
    if (!d) return fail(SAIS_EINVAL, "descriptor is NULL");
    if (d->n < 1) return fail(SAIS_EINVAL, "n = %d: need at least one item", d->n);
    if (d->m < 0 || d->m > kMaxConstraints)
        return fail(SAIS_EINVAL, "m = %d: need 0 <= m <= %d", d->m, kMaxConstraints);
    if (!d->h) return fail(SAIS_EINVAL, "h is NULL");
    if (d->m > 0 && (!d->A || !d->b)) return fail(SAIS_EINVAL, "A or b is NULL with m > 0");
    if (!std::isfinite(d->alpha) || !std::isfinite(d->density) || !std::isfinite(d->penalty))
        return fail(SAIS_EINVAL, "alpha, density and penalty must be finite");
    const int32_t n = d->n, m = d->m;
    h.n = n;
    h.m = m;
    h.has_w = d->W != nullptr;
    h.W = d->W;

    // Integer checks: W symmetric with zero diagonal and int16 range; A >= 0; b >= 1.
    int64_t maxabs_f = 0, nz = 0, max_w = 0, max_row = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t row = std::llabs((int64_t)d->h[i]);
        maxabs_f = std::max(maxabs_f, row);
        if (d->h[i] != 0) ++nz;
        if (h.has_w) {
            for (int32_t j = 0; j < n; ++j) {
                const int32_t w = d->W[(size_t)i * n + j];
                if (w != d->W[(size_t)j * n + i])
                    return fail(SAIS_EINVAL, "W is not symmetric at (%d,%d)", i, j);
                if (i == j && w != 0) return fail(SAIS_EINVAL, "W has nonzero diagonal at %d", i);
                if (w > 32767 || w < -32767)
                    return fail(SAIS_EOVERFLOW, "|W(%d,%d)| = %d exceeds 32767", i, j, w);
                const int64_t aw = std::llabs((int64_t)w);
                maxabs_f = std::max(maxabs_f, aw);
                max_w = std::max(max_w, aw);
                row += aw;
                if (j > i && w != 0) ++nz;
            }
        }
        if (row >= kExact24)
            return fail(SAIS_EOVERFLOW,
                        "item %d: |h| + sum |W| = %lld >= 2^24 breaks the exact FP32 field", i,
                        (long long)row);
        max_row = std::max(max_row, row);
    }
    h.need_lo = max_w > 256;
    h.f16 = h.has_w && max_row <= 32767;   // |F_i| <= max_row for every state
    h.lo_own = h.need_lo;
    // Capacity tightening (Sec. IV-B): the sampled problem uses B' (slack bits, sigma_g, g,
    // penalty rule); feasibility keeps the caller's b through a per-constraint margin.
    const int64_t *bs = d->b_tight ? d->b_tight : d->b;
    int64_t maxabs_g = 0;
    h.Q.assign(m, 0);
    h.margin.assign(m, 0);
    h.slack_off.assign(m + 1, 0);
    int32_t nprime = n;
    for (int32_t k = 0; k < m; ++k) {
        const int64_t bk = bs[k];
        if (d->b[k] < 1) return fail(SAIS_EINVAL, "b[%d] = %lld: capacities must be >= 1", k, (long long)d->b[k]);
        if (bk < 1 || bk > d->b[k])
            return fail(SAIS_EINVAL, "b_tight[%d] = %lld: need 1 <= b_tight <= b = %lld", k,
                        (long long)bk, (long long)d->b[k]);
        int64_t rowsum = 0;
        for (int32_t i = 0; i < n; ++i) {
            const int32_t a = d->A[(size_t)k * n + i];
            if (a < 0) return fail(SAIS_EINVAL, "A(%d,%d) = %d is negative", k, i, a);
            rowsum += a;
            maxabs_g = std::max(maxabs_g, (int64_t)a);
        }
        maxabs_g = std::max(maxabs_g, bk);
        // items load l <= b  <=>  l - B' <= b - B'; the load never exceeds the row sum, so the
        // margin is capped there (it then fits int32)
        h.margin[k] = (int32_t)std::min<int64_t>(d->b[k] - bk, rowsum);
        h.Q[k] = binary_digits(bk);
        h.slack_off[k] = nprime;
        nprime += h.Q[k];
        // |g_k| <= max(b_k, sum_i a_ki + 2^Q - 1 - b_k) must stay exact in FP32 / int32
        const int64_t span = rowsum + ((int64_t(1) << h.Q[k]) - 1) + bk;
        if (span >= kExact24)
            return fail(SAIS_EOVERFLOW,
                        "constraint %d: b + sum a + slack range = %lld >= 2^24", k,
                        (long long)span);
    }
    h.slack_off[m] = nprime;
    h.nprime = nprime;
    h.npad = (nprime + kSpinPad - 1) / kSpinPad * kSpinPad;
    h.words = (nprime + 31) / 32;

    // Scalars (Sec. III-A, IV-A, IV-B), each rounded once to FP32.
    h.sf = maxabs_f > 0 ? (float)(1.0 / (double)maxabs_f) : 1.0f;
    h.sg = maxabs_g > 0 ? (float)(1.0 / (double)maxabs_g) : 1.0f;
    if (d->density >= 0.0f)
        h.d = (double)d->density;
    else if (!h.has_w)
        h.d = 2.0 / ((double)nprime + 1.0);
    else
        h.d = (double)nz / (0.5 * (double)n * (double)(n + 1));
    h.P = d->penalty > 0.0f ? d->penalty : (float)((double)d->alpha * h.d * (double)nprime);
    if (!(h.P >= 0.0f) || !std::isfinite(h.P)) return fail(SAIS_EINVAL, "penalty P is negative or not finite");
    h.psg2 = (double)h.P * (double)h.sg * (double)h.sg;
    h.kappa = (float)(2.0 * h.psg2);

    // Spin-major constraint columns of A_ext, D_i and sum_k a_ki, zero-padded to N'_pad spins
    // (kernels may read whole blocks of spins).
    h.acol.assign((size_t)h.npad * std::max(m, 1), 0);
    h.D.assign(h.npad, 0.f);
    h.asum.assign(h.npad, 0.f);
    h.b.assign(m, 0);
    for (int32_t k = 0; k < m; ++k) {
        h.b[k] = (int32_t)bs[k];
        for (int32_t i = 0; i < n; ++i) h.acol[(size_t)i * m + k] = d->A[(size_t)k * n + i];
        for (int32_t q = 0; q < h.Q[k]; ++q)
            h.acol[(size_t)(h.slack_off[k] + q) * m + k] = 1 << q;
    }
    for (int32_t i = 0; i < nprime; ++i) {
        int64_t s2 = 0, s1 = 0;
        for (int32_t k = 0; k < m; ++k) {
            const int64_t a = h.acol[(size_t)i * m + k];
            s2 += a * a;
            s1 += a;
        }
        h.D[i] = (float)(h.psg2 * (double)s2);
        h.asum[i] = (float)s1;
    }
    h.spinc.assign((size_t)h.npad * 4, 0.f);
    for (int32_t i = 0; i < nprime; ++i) {
        h.spinc[(size_t)i * 4 + 0] = m > 0 ? (float)h.acol[(size_t)i * m] : 0.f;
        h.spinc[(size_t)i * 4 + 1] = h.D[i];
        h.spinc[(size_t)i * 4 + 2] = h.asum[i];
        h.spinc[(size_t)i * 4 + 3] = m > 1 ? (float)h.acol[(size_t)i * m + 1] : 0.f;
    }
    h.hF.assign(h.npad, 0.f);
    for (int32_t i = 0; i < n; ++i) h.hF[i] = (float)d->h[i];

    // Features of the warm-start network (one row per constraint): capacity ratio, weight
    // statistics in sigma_g units, profit statistics in sigma_f units, size and density.
    double psum = 0.0, psq = 0.0, pcnt = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        const double hv = (double)d->h[i];
        if (hv != 0.0) {
            psum += hv;
            psq += hv * hv;
            pcnt += 1.0;
        }
        if (h.has_w)
            for (int32_t j = i + 1; j < n; ++j) {
                const double wv = (double)d->W[(size_t)i * n + j];
                if (wv != 0.0) {
                    psum += wv;
                    psq += wv * wv;
                    pcnt += 1.0;
                }
            }
    }
    const double pmu = pcnt > 0.0 ? psum / pcnt : 0.0;
    const double pvar = pcnt > 0.0 ? psq / pcnt - pmu * pmu : 0.0;
    h.feat.assign((size_t)m * 8, 0.f);
    for (int32_t k = 0; k < m; ++k) {
        double as = 0.0, asq = 0.0;
        for (int32_t i = 0; i < n; ++i) {
            const double av = (double)d->A[(size_t)k * n + i];
            as += av;
            asq += av * av;
        }
        const double amu = as / n, avar = asq / n - amu * amu;
        float *f = &h.feat[(size_t)k * 8];
        f[0] = (float)(as > 0.0 ? std::min(1.0, (double)bs[k] / as) : 1.0);
        f[1] = (float)((double)h.sg * amu);
        f[2] = (float)((double)h.sg * std::sqrt(std::max(avar, 0.0)));
        f[3] = (float)((double)h.sf * pmu);
        f[4] = (float)((double)h.sf * std::sqrt(std::max(pvar, 0.0)));
        f[5] = (float)(n / 1000.0);
        f[6] = (float)h.d;
    }
    return SAIS_OK;
}

uint16_t bf16_bits(float f) {  // f is an integer of magnitude < 2^16: round to nearest even
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}

float bf16_value(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int32_t n16_of(int32_t n) { return (n + 15) / 16 * 16; }

struct DeviceGuard {
    int prev = 0;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        cudaSetDevice(dev);
    }
    ~DeviceGuard() { cudaSetDevice(prev); }
};

}  // namespace

struct sais_problem {
    int device = 0;
    int count = 0;
    int max_spins = 0, max_npad = 0, max_npad_w = 0, words = 0, m_stride = 1, max_m = 0;
    int max_n = 0;
    int max_n16 = 0;              // max over quadratic instances of n rounded up to 16
    bool any_w = false;
    bool all_f16 = true;          // every quadratic instance has HostInst::f16
    std::vector<HostInst> host;   // host copies (W pointer cleared after creation)
    bool any_lo = false;          // some instance needs the BF16 hi/lo split
    bool all_w = true;            // every instance has a quadratic objective
    void *pool = nullptr;         // one device allocation for all instance arrays
    InstDev *d_inst = nullptr;    // device array of count records (inside pool)
    int32_t *d_status = nullptr;  // device status word written by kernels (inside pool)
    int32_t feat_rows = 0;        // sum of m over the instances
    float *d_feat = nullptr;      // feat_rows x 8 warm-start features (inside pool)
    int32_t *d_feat_dst = nullptr;   // row -> j m_stride + k (inside pool)

    // Launch groups of SAIS_AUTO: instances the blocked sampler runs, grouped by how it holds W
    // (resident, streamed, streamed hi/lo), and the rest on the plain sampler.  Members are kept
    // most expensive first; each group runs over a slice of a device work list of (instance,
    // chain group) pairs, so the block scheduler starts the longest work first.
    struct Group {
        int variant = SAIS_PLAIN;
        bool stream_w = false, hilo = false;
        int block_k = 16, cpb = 32;
        int max_m = 0, max_npad = 0, max_npad_w = 0, words = 0, max_n = 0, max_n16 = 0;
        bool any_w = false;
        bool f16 = true;           // every quadratic member has HostInst::f16 (plain: int16 F)
        bool blocked_ok = false;   // every member fits the blocked sampler
        bool field = false;        // blocked sampler with per-block field GEMMs (one CTA)
        std::vector<int> members;
        size_t work_off = 0, nwork = 0;
        double tuned_ms = 0.0;
    };
    std::vector<Group> groups;
    std::vector<int32_t> inst_chains;   // chains per instance (empty: one count for all)
    int32_t *d_inst_chains = nullptr;   // device copy (own allocation)
    int32_t *d_work = nullptr;          // device work list (own allocation)
    // Launch groups run concurrently: fork from the caller's stream, one side stream per group
    // (the extra stream side[0] is spare), join back.
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    size_t work_cap = 0;                // capacity in (instance, group) pairs
    int work_chains = -1;               // `chains` the work list was built for
    bool work_valid = false;
    int32_t *h_work = nullptr;          // pinned staging copy of the work list (own allocation)
    cudaEvent_t work_copied = nullptr;  // the last upload from h_work has completed
    // The persistent launch of SAIS_AUTO (sais_ragged_kernel.cuh): its items follow the group
    // pairs in the work list, 3 ints each (instance, chain group, kind), most expensive first,
    // then the device work counter.
    bool ragged_ok = false;             // every instance fits the persistent launch
    bool use_ragged = false;            // SAIS_AUTO runs it (else the per-group launches)
    size_t ragged_off = 0, ragged_n = 0, head_off = 0;   // in ints of the work list
    size_t stats_off = 0;   // per-CTA records of the persistent launch (4 uint64 per CTA)
    int ragged_ctas = 0;    // CTAs of the persistent launch
    int sms = 0;                        // multiprocessors of the device
};

namespace {

// The blocked samplers, by instance size (N'_pad spins, n items):
//  * rank-k update with every field resident in TMEM (sais_blocked_kernel.cuh), one CTA per SM:
//    N'_pad + K <= 512; two MMAs per block of K = 16 spins, the fewest tensor-core
//    instructions per spin;
//  * block fields from a GEMM over the states (sais_field_kernel.cuh), one CTA per SM up to
//    n = 1024 items: for instances beyond the first, and for K = 32 streamed or hi/lo and K = 64.
bool field_fits(int n16, int words, int m, bool has_w, int k, bool hilo) {
    return has_w && m <= kMaxBlockedConstraints && (k == 16 || m <= 2) && n16 <= 1024 &&
           field_smem_bytes(n16, words, k, hilo) <= kMaxSmemPerBlock;
}

// The block size of the block-field sampler when the caller leaves it open: 32 (half the MMA
// instructions per spin of K = 16, measured faster at n = 500 and 900) where m <= 2 allows it.
int field_default_k(int m) { return m <= 2 ? 32 : 16; }

// SAIS_AUTO grouping (see struct sais_problem).  Keys: 1 rank-k blocked with W resident, 2
// streamed, 3 streamed hi/lo; 10 block-field, 11 block-field hi/lo; plain instances split by
// whether they have W and by padded N' (bucket of 128 spins), so each plain group sizes its
// shared memory for its own largest member.

void build_groups(sais_problem *p) {
    p->groups.clear();
    auto key_of = [&](const HostInst &h) -> int {
        const bool eligible = h.has_w && h.m <= kMaxBlockedConstraints && h.npad + 16 <= 512;
        if (eligible) {
            if (h.lo_own) return 3;
            return blocked_smem_bytes(h.npad, h.words, 16, false, false) > kMaxSmemPerBlock ? 2 : 1;
        }
        if (field_fits(n16_of(h.n), h.words, h.m, h.has_w, 16, h.lo_own))
            return h.lo_own ? 11 : 10;
        return 100 + (h.has_w ? 1000 : 0) + (h.npad + 127) / 128;
    };
    std::vector<int> keys;
    for (int j = 0; j < p->count; ++j) keys.push_back(key_of(p->host[j]));
    std::vector<int> uniq = keys;
    std::sort(uniq.begin(), uniq.end());
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    // blocked groups first (ascending key), then plain groups, largest N' first
    std::stable_sort(uniq.begin(), uniq.end(), [](int x, int y) {
        const bool bx = x < 100, by = y < 100;
        if (bx != by) return bx;
        return bx ? x < y : x > y;
    });
    for (int key : uniq) {
        sais_problem::Group g;
        for (int j = 0; j < p->count; ++j) {
            if (keys[j] != key) continue;
            const HostInst &h = p->host[j];
            g.members.push_back(j);
            g.max_m = std::max(g.max_m, h.m);
            g.max_npad = std::max(g.max_npad, h.npad);
            g.max_n = std::max(g.max_n, h.n);
            g.max_n16 = std::max(g.max_n16, n16_of(h.n));
            if (h.has_w) g.max_npad_w = std::max(g.max_npad_w, h.npad);
            g.words = std::max(g.words, h.words);
            g.any_w = g.any_w || h.has_w;
            if (h.has_w) g.f16 = g.f16 && h.f16;
        }
        g.variant = key >= 100 ? SAIS_PLAIN : SAIS_BLOCKED;
        g.blocked_ok = key < 100;
        g.field = key == 10 || key == 11;
        g.stream_w = key >= 2 && key <= 11;
        g.hilo = key == 3 || key == 11;
        if (g.field) {   // the default block size where the group's largest member fits it
            g.block_k = field_default_k(g.max_m);
            if (!field_fits(g.max_n16, g.words, g.max_m, true, g.block_k, g.hilo)) g.block_k = 16;
        }
        auto cost = [&](int j) {
            const HostInst &h = p->host[j];
            return (double)h.nprime * (h.has_w ? (double)h.npad : (double)std::max(1, h.m));
        };
        std::stable_sort(g.members.begin(), g.members.end(),
                         [&](int x, int y) { return cost(x) > cost(y); });
        p->groups.push_back(std::move(g));
    }
    p->work_valid = false;
    // The persistent launch: quadratic instances on the block-field sampler (m <= 8, n <= 1024),
    // linear ones on the plain sampler (m <= 32), the whole batch's shared memory in one CTA.
    p->ragged_ok = p->count > 0;
    int max_n16_w = 0;
    for (const HostInst &h : p->host) {
        if (h.has_w) {
            max_n16_w = std::max(max_n16_w, n16_of(h.n));
            p->ragged_ok = p->ragged_ok && h.m <= kMaxBlockedConstraints && n16_of(h.n) <= 1024;
        } else {
            p->ragged_ok = p->ragged_ok && h.m <= kMaxConstraints;
        }
    }
    int ring = 0;
    p->ragged_ok = p->ragged_ok &&
                   ragged_smem_bytes(max_n16_w, p->words, p->any_lo, &ring) <= kMaxSmemPerBlock;
    p->use_ragged = p->ragged_ok;
    if (p->groups.size() > 1) {
        const size_t ns = p->groups.size() + 1;
        p->side.assign(ns, nullptr);
        p->join.assign(ns, nullptr);
        for (size_t i = 0; i < ns; ++i) {
            cudaStreamCreateWithFlags(&p->side[i], cudaStreamNonBlocking);
            cudaEventCreateWithFlags(&p->join[i], cudaEventDisableTiming);
        }
        cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
    }
}

int group_cta(const sais_problem::Group &g) { return g.variant == SAIS_BLOCKED ? 128 : g.cpb; }

// Device work list for `chains` (the uniform count, or the stride when per-instance counts are
// set).  Built on the host and uploaded asynchronously on the caller's stream from a pinned
// staging buffer, so the sampling path does not block the host: launches queued before it on
// that stream (every group joins back into it) still read the old list, later ones the new one.
// The host waits only when the staging buffer's previous upload is still in flight, or when
// the list outgrows its allocation (cudaFree synchronises the device).  Refused during capture.
sais_status ensure_work(sais_problem *p, int chains, cudaStream_t st) {
    if (p->work_valid && p->work_chains == chains) return SAIS_OK;
    std::vector<int32_t> w;
    for (auto &g : p->groups) {
        g.work_off = w.size() / 2;
        const int cta = group_cta(g);
        for (int j : g.members) {
            const int cj = p->inst_chains.empty() ? chains : p->inst_chains[j];
            for (int q = 0; q < (cj + cta - 1) / cta; ++q) {
                w.push_back(j);
                w.push_back(q);
            }
        }
        g.nwork = w.size() / 2 - g.work_off;
    }
    if (p->ragged_ok) {
        // Items of the persistent launch, most expensive first by an estimate of SM cycles per
        // sweep: the block-field sampler ~150 per spin plus ~7.5 per spin for each 16-spin
        // GEMM step (one MMA per step, hi/lo included); the plain sampler on 256 chains
        // ~(120 + 6 m) per spin.
        struct Item {
            double cost;
            int32_t j, q, kind;
        };
        std::vector<Item> items;
        for (int j = 0; j < p->count; ++j) {
            const HostInst &h = p->host[j];
            const int cj = p->inst_chains.empty() ? chains : p->inst_chains[j];
            const int per = h.has_w ? kRaggedFieldChains : kRaggedPlainItemChains;
            const int kind = h.has_w ? (h.m <= 1 ? 0 : 1) : (h.m <= 8 ? 2 : 3);
            const double cost =
                h.has_w ? (double)h.nprime * (150.0 + 7.5 * (n16_of(h.n) / 16))
                        : (double)h.nprime * (120.0 + 6.0 * h.m);
            for (int q = 0; q < (cj + per - 1) / per; ++q) items.push_back({cost, j, q, kind});
        }
        std::stable_sort(items.begin(), items.end(),
                         [](const Item &x, const Item &y) { return x.cost > y.cost; });
        p->ragged_off = w.size();
        p->ragged_n = items.size();
        for (const Item &it : items) {
            w.push_back(it.j);
            w.push_back(it.q);
            w.push_back(it.kind);
        }
        while (w.size() % 64) w.push_back(0);   // the counter on its own 256 bytes
        p->head_off = w.size();
        for (int i = 0; i < 64; ++i) w.push_back(0);
        p->stats_off = w.size();
        p->ragged_ctas = ragged_grid((int)items.size(), p->sms);
        for (int i = 0; i < 8 * p->ragged_ctas; ++i) w.push_back(0);
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs != cudaStreamCaptureStatusNone)
        return fail(SAIS_EINVAL, "SAIS_AUTO: prepare the launch (one call with these chains) "
                                 "before capturing a graph");
    cudaError_t e = cudaSuccess;
    if (!p->work_copied) {
        e = cudaEventCreateWithFlags(&p->work_copied, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(SAIS_ECUDA, "work list event: %s", cudaGetErrorString(e));
    }
    if (w.size() / 2 > p->work_cap) {
        if (p->d_work) {   // synchronise first: queued launches may still read it
            cudaDeviceSynchronize();
            dev_free(p->d_work);
        }
        if (p->h_work) cudaFreeHost(p->h_work);
        p->d_work = nullptr;
        p->h_work = nullptr;
        p->work_cap = 0;
        e = dev_alloc(reinterpret_cast<void **>(&p->d_work), w.size() * 4);
        if (e != cudaSuccess) return fail(SAIS_ENOMEM, "work list: %s", cudaGetErrorString(e));
        e = cudaMallocHost(&p->h_work, w.size() * 4);
        if (e != cudaSuccess) return fail(SAIS_ENOMEM, "work list staging: %s", cudaGetErrorString(e));
        p->work_cap = w.size() / 2;
    } else {
        e = cudaEventSynchronize(p->work_copied);   // the staging buffer's last upload is done
        if (e != cudaSuccess) return fail(SAIS_ECUDA, "work list: %s", cudaGetErrorString(e));
    }
    std::memcpy(p->h_work, w.data(), w.size() * 4);
    e = cudaMemcpyAsync(p->d_work, p->h_work, w.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(p->work_copied, st);
    if (e != cudaSuccess) return fail(SAIS_ECUDA, "work list copy: %s", cudaGetErrorString(e));
    p->work_chains = chains;
    p->work_valid = true;
    return SAIS_OK;
}

cudaError_t launch_group(const sais_problem *p, const sais_problem::Group &g, const SampleArgs &a,
                         long long polls, cudaStream_t st) {
    if (g.nwork == 0) return cudaSuccess;
    SampleArgs ga = a;
    ga.work = p->d_work + 2 * g.work_off;
    ga.nwork = (int32_t)g.nwork;
    if (g.variant == SAIS_BLOCKED && g.field)
        return launch_field_sampler(ga, g.max_m, g.max_n16, g.words, g.block_k, g.hilo,
                                    p->d_status, polls, st);
    if (g.variant == SAIS_BLOCKED)
        return launch_blocked_sampler(ga, g.max_m, g.max_npad, g.words, g.block_k, g.stream_w,
                                      g.hilo, p->d_status, polls, st);
    return launch_plain_sampler(ga, g.max_m, g.max_npad_w, g.words, g.cpb, st, g.f16);
}

}  // namespace

extern "C" {

const char *sais_status_string(sais_status s) {
    switch (s) {
        case SAIS_OK: return "ok";
        case SAIS_EINVAL: return "invalid argument";
        case SAIS_ENOMEM: return "out of memory";
        case SAIS_ECUDA: return "CUDA error";
        case SAIS_EOVERFLOW: return "integer bound for exact fields exceeded";
        case SAIS_ETIMEOUT: return "bounded device wait timed out";
        case SAIS_EUNSUPPORTED: return "unsupported device or size";
        case SAIS_EBOUNDS: return "device-side bounds check failed (debug build)";
    }
    return "unknown status";
}

const char *sais_last_error(void) { return g_last_error.c_str(); }

sais_status sais_describe(const sais_problem_desc *desc, sais_problem_scalars *out) {
    if (!out) return fail(SAIS_EINVAL, "out is NULL");
    HostInst h;
    sais_status s = build_host(desc, h);
    if (s != SAIS_OK) return s;
    out->n = h.n;
    out->m = h.m;
    out->n_spins = h.nprime;
    out->words = h.words;
    out->sigma_f = h.sf;
    out->sigma_g = h.sg;
    out->penalty = h.P;
    out->reserved = 0.f;
    out->density = h.d;
    return SAIS_OK;
}

sais_status sais_create_batch(const sais_problem_desc *descs, int32_t count, int32_t device,
                              sais_problem **out) {
    NvtxRange nvtx_range("sais_create_batch");
    if (!out) return fail(SAIS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!descs || count < 1) return fail(SAIS_EINVAL, "need count >= 1 descriptors");
    if (count > 65535) return fail(SAIS_EUNSUPPORTED, "count = %d: at most 65535 instances", count);
    int ndev = 0;
    SAIS_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev)
        return fail(SAIS_EINVAL, "device %d out of range (%d devices)", device, ndev);
    cudaDeviceProp prop;
    SAIS_CUDA(cudaGetDeviceProperties(&prop, device));
    if (!(prop.major == 10 && prop.minor == 3))
        return fail(SAIS_EUNSUPPORTED, "device %d is sm_%d%d; libsais is built for sm_103a",
                    device, prop.major, prop.minor);

    sais_problem *p = new (std::nothrow) sais_problem;
    if (!p) return fail(SAIS_ENOMEM, "host allocation failed");
    p->device = device;
    p->count = count;
    p->host.resize(count);
    for (int32_t j = 0; j < count; ++j) {
        sais_status s = build_host(descs + j, p->host[j]);
        if (s != SAIS_OK) {
            std::string msg = g_last_error;
            delete p;
            return fail(s, "instance %d: %s", j, msg.c_str());
        }
        const HostInst &h = p->host[j];
        p->max_spins = std::max(p->max_spins, h.nprime);
        p->max_npad = std::max(p->max_npad, h.npad);
        p->max_n = std::max(p->max_n, h.n);
        if (h.has_w) {
            p->max_npad_w = std::max(p->max_npad_w, h.npad);
            p->max_n16 = std::max(p->max_n16, n16_of(h.n));
        }
        p->max_m = std::max(p->max_m, h.m);
        p->any_w = p->any_w || h.has_w;
        if (h.has_w) p->all_f16 = p->all_f16 && h.f16;
        p->all_w = p->all_w && h.has_w;
        p->any_lo = p->any_lo || h.need_lo;
    }
    p->words = (p->max_spins + 31) / 32;
    p->m_stride = std::max(1, p->max_m);

    // Pool layout: [InstDev x count] then per instance W, Wbf(, Wbf_lo), hF, acol, D, asum, b,
    // slack_off, each 256-byte aligned.
    struct Off {
        size_t W, Wbf, Wlo, Wd, Wg, Wglo, Wd32, Wd64, hF, acol, acf, D, asum, spinc, b, so;
    };
    int32_t feat_rows = 0;
    for (const HostInst &h : p->host) feat_rows += h.m;
    std::vector<Off> off(count);
    // In a batch with any pair value above 256 every instance gets a lo image (zero where the
    // hi term is already exact), since one launch serves the whole batch.
    if (p->any_lo)
        for (HostInst &h : p->host)
            if (h.has_w) h.need_lo = true;
    size_t cur = align_up(sizeof(InstDev) * count, 256);
    const size_t status_off = cur;
    cur = align_up(cur + 4, 256);
    for (int32_t j = 0; j < count; ++j) {
        const HostInst &h = p->host[j];
        const size_t nn = (size_t)h.npad * h.npad;
        Off &o = off[j];
        o.W = o.Wbf = o.Wlo = o.Wd = o.Wg = o.Wglo = o.Wd32 = o.Wd64 = SIZE_MAX;
        if (h.has_w) {
            const size_t ng = (size_t)h.npad * n16_of(h.n);
            o.W = cur;
            cur = align_up(cur + nn * 2, 256);
            o.Wd = cur;
            cur = align_up(cur + (size_t)h.npad * 16 * 4, 256);
            o.Wd32 = cur;
            cur = align_up(cur + (size_t)h.npad * 32 * 4, 256);
            o.Wd64 = cur;
            cur = align_up(cur + (size_t)h.npad * 64 * 4, 256);
            o.Wbf = cur;
            cur = align_up(cur + nn * 2, 256);
            o.Wg = cur;
            cur = align_up(cur + ng * 2, 256);
            if (h.need_lo) {
                o.Wlo = cur;
                cur = align_up(cur + nn * 2, 256);
                o.Wglo = cur;
                cur = align_up(cur + ng * 2, 256);
            }
        }
        o.hF = cur;
        cur = align_up(cur + (size_t)h.npad * 4, 256);
        o.acol = cur;
        cur = align_up(cur + h.acol.size() * 4, 256);
        o.acf = cur;
        cur = align_up(cur + (size_t)h.npad * ((h.m + 3) / 4 * 4) * 4, 256);
        o.D = cur;
        cur = align_up(cur + h.D.size() * 4, 256);
        o.asum = cur;
        cur = align_up(cur + h.asum.size() * 4, 256);
        o.spinc = cur;
        cur = align_up(cur + h.spinc.size() * 4, 256);
        o.b = cur;   // b, then the feasibility margins
        cur = align_up(cur + (size_t)std::max(h.m, 1) * 8, 256);
        o.so = cur;
        cur = align_up(cur + (size_t)(h.m + 1) * 4, 256);
    }
    const size_t feat_off = cur;
    cur = align_up(cur + (size_t)std::max(feat_rows, 1) * 8 * 4, 256);
    const size_t dst_off = cur;
    cur = align_up(cur + (size_t)std::max(feat_rows, 1) * 4, 256);
    std::vector<unsigned char> stage;
    try {
        stage.assign(cur, 0);
    } catch (...) {
        delete p;
        return fail(SAIS_ENOMEM, "host staging allocation of %zu bytes failed", cur);
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    cudaError_t ce = dev_alloc(&p->pool, cur);
    if (ce != cudaSuccess) {
        cudaSetDevice(prev);
        delete p;
        return fail(ce == cudaErrorMemoryAllocation ? SAIS_ENOMEM : SAIS_ECUDA,
                    "device allocation of %zu bytes: %s", cur, cudaGetErrorString(ce));
    }
    unsigned char *base = static_cast<unsigned char *>(p->pool);
    InstDev *recs = reinterpret_cast<InstDev *>(stage.data());
    for (int32_t j = 0; j < count; ++j) {
        HostInst &h = p->host[j];
        const Off &o = off[j];
        InstDev r{};
        r.n = h.n;
        r.m = h.m;
        r.nprime = h.nprime;
        r.npad = h.npad;
        r.words = h.words;
        r.n16 = n16_of(h.n);
        r.has_w = h.has_w ? 1 : 0;
        r.sigma_f = h.sf;
        r.sigma_g = h.sg;
        r.P = h.P;
        r.kappa = h.kappa;
        r.psg2 = h.psg2;
        if (h.has_w) {
            int16_t *W16 = reinterpret_cast<int16_t *>(stage.data() + o.W);
            uint16_t *Wb = reinterpret_cast<uint16_t *>(stage.data() + o.Wbf);
            uint16_t *Wl = h.need_lo ? reinterpret_cast<uint16_t *>(stage.data() + o.Wlo) : nullptr;
            for (int32_t i = 0; i < h.n; ++i)
                for (int32_t jj = 0; jj < h.n; ++jj) {
                    const int32_t w = h.W[(size_t)i * h.n + jj];
                    W16[(size_t)i * h.npad + jj] = (int16_t)w;
                    // shared-memory image of the blocked sampler: element (row i, column jj)
                    // at ((jj/8) npad + i) 8 + jj%8
                    const size_t e = ((size_t)(jj >> 3) * h.npad + i) * 8 + (jj & 7);
                    const uint16_t hi = bf16_bits((float)w);
                    Wb[e] = hi;
                    if (Wl) Wl[e] = bf16_bits((float)w - bf16_value(hi));
                }
            // Block-field image: element (i, jj) at ((i/8)(n16/8) + jj/8) 64 + (i%8) 8 + jj%8.
            const int32_t n16 = n16_of(h.n);
            uint16_t *Wg = reinterpret_cast<uint16_t *>(stage.data() + o.Wg);
            uint16_t *Wgl = h.need_lo ? reinterpret_cast<uint16_t *>(stage.data() + o.Wglo) : nullptr;
            for (int32_t i = 0; i < h.n; ++i)
                for (int32_t jj = 0; jj < h.n; ++jj) {
                    const int32_t w = h.W[(size_t)i * h.n + jj];
                    const size_t e = ((size_t)(i >> 3) * (n16 >> 3) + (jj >> 3)) * 64 +
                                     (size_t)(i & 7) * 8 + (jj & 7);
                    const uint16_t hi = bf16_bits((float)w);
                    Wg[e] = hi;
                    if (Wgl) Wgl[e] = bf16_bits((float)w - bf16_value(hi));
                }
            // FP32 diagonal blocks of W for block sizes 16, 32 and 64 (row-major per block).
            const size_t doff[3] = {o.Wd, o.Wd32, o.Wd64};
            for (int q = 0; q < 3; ++q) {
                const int32_t kb = 16 << q;
                float *Wd = reinterpret_cast<float *>(stage.data() + doff[q]);
                for (int32_t i = 0; i < h.n; ++i)
                    for (int32_t jj = (i / kb) * kb; jj < std::min(h.n, (i / kb) * kb + kb); ++jj)
                        Wd[(size_t)(i / kb) * kb * kb + (size_t)(i % kb) * kb + (jj % kb)] =
                            (float)h.W[(size_t)i * h.n + jj];
            }
            r.Wdiag = reinterpret_cast<const float *>(base + o.Wd);
            r.Wd32 = reinterpret_cast<const float *>(base + o.Wd32);
            r.Wd64 = reinterpret_cast<const float *>(base + o.Wd64);
            r.Wg = reinterpret_cast<const uint16_t *>(base + o.Wg);
            r.Wg_lo = h.need_lo ? reinterpret_cast<const uint16_t *>(base + o.Wglo) : nullptr;
            r.W = reinterpret_cast<const int16_t *>(base + o.W);
            r.Wbf = reinterpret_cast<const uint16_t *>(base + o.Wbf);
            r.Wbf_lo = h.need_lo ? reinterpret_cast<const uint16_t *>(base + o.Wlo) : nullptr;
        }
        std::memcpy(stage.data() + o.hF, h.hF.data(), h.hF.size() * 4);
        std::memcpy(stage.data() + o.acol, h.acol.data(), h.acol.size() * 4);
        {
            const int m4 = (h.m + 3) / 4 * 4;
            float *af = reinterpret_cast<float *>(stage.data() + o.acf);
            for (int32_t i = 0; i < h.npad; ++i)
                for (int32_t k = 0; k < h.m; ++k)
                    af[(size_t)i * m4 + k] = (float)h.acol[(size_t)i * h.m + k];
            r.acf = reinterpret_cast<const float *>(base + o.acf);
            r.m4 = m4;
        }
        std::memcpy(stage.data() + o.D, h.D.data(), h.D.size() * 4);
        std::memcpy(stage.data() + o.asum, h.asum.data(), h.asum.size() * 4);
        std::memcpy(stage.data() + o.spinc, h.spinc.data(), h.spinc.size() * 4);
        if (h.m) {
            std::memcpy(stage.data() + o.b, h.b.data(), h.b.size() * 4);
            std::memcpy(stage.data() + o.b + (size_t)h.m * 4, h.margin.data(), h.margin.size() * 4);
        }
        std::memcpy(stage.data() + o.so, h.slack_off.data(), h.slack_off.size() * 4);
        r.hF = reinterpret_cast<const float *>(base + o.hF);
        r.acol = reinterpret_cast<const int32_t *>(base + o.acol);
        r.D = reinterpret_cast<const float *>(base + o.D);
        r.asum = reinterpret_cast<const float *>(base + o.asum);
        r.spinc = reinterpret_cast<const float4 *>(base + o.spinc);
        r.b = reinterpret_cast<const int32_t *>(base + o.b);
        r.fmargin = reinterpret_cast<const int32_t *>(base + o.b) + h.m;
        r.slack_off = reinterpret_cast<const int32_t *>(base + o.so);
        recs[j] = r;
        h.W = nullptr;
    }
    {
        float *F = reinterpret_cast<float *>(stage.data() + feat_off);
        int32_t *Dst = reinterpret_cast<int32_t *>(stage.data() + dst_off);
        int32_t r = 0;
        for (int32_t j = 0; j < count; ++j)
            for (int32_t k = 0; k < p->host[j].m; ++k, ++r) {
                std::memcpy(F + (size_t)r * 8, &p->host[j].feat[(size_t)k * 8], 8 * 4);
                Dst[r] = j * p->m_stride + k;
            }
    }
    p->feat_rows = feat_rows;
    p->d_feat = reinterpret_cast<float *>(base + feat_off);
    p->d_feat_dst = reinterpret_cast<int32_t *>(base + dst_off);
    ce = cudaMemcpy(p->pool, stage.data(), cur, cudaMemcpyHostToDevice);
    cudaSetDevice(prev);
    if (ce != cudaSuccess) {
        dev_free(p->pool);
        delete p;
        return fail(SAIS_ECUDA, "copy of problem data: %s", cudaGetErrorString(ce));
    }
    p->d_inst = reinterpret_cast<InstDev *>(p->pool);
    p->d_status = reinterpret_cast<int32_t *>(base + status_off);
    {
        DeviceGuard dg(device);   // the groups' side streams belong to the problem's device
        cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, device);
        build_groups(p);
    }
    noalloc_prepare(device);
    *out = p;
    return SAIS_OK;
}

sais_status sais_create_problem(const sais_problem_desc *desc, int32_t device,
                                sais_problem **out) {
    return sais_create_batch(desc, 1, device, out);
}

sais_status sais_destroy_problem(sais_problem *p) {
    if (!p) return SAIS_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (p->pool) dev_free(p->pool);
    if (p->d_work) dev_free(p->d_work);
    if (p->h_work) cudaFreeHost(p->h_work);
    if (p->work_copied) cudaEventDestroy(p->work_copied);
    if (p->d_inst_chains) dev_free(p->d_inst_chains);
    for (cudaStream_t x : p->side)
        if (x) cudaStreamDestroy(x);
    for (cudaEvent_t x : p->join)
        if (x) cudaEventDestroy(x);
    if (p->fork) cudaEventDestroy(p->fork);
    cudaSetDevice(prev);
    delete p;
    if (e != cudaSuccess) return fail(SAIS_ECUDA, "synchronize before free: %s", cudaGetErrorString(e));
    return SAIS_OK;
}

sais_status sais_problem_info(const sais_problem *p, sais_layout *out) {
    if (!p || !out) return fail(SAIS_EINVAL, "NULL argument");
    out->count = p->count;
    out->max_spins = p->max_spins;
    out->words = p->words;
    out->m_stride = p->m_stride;
    out->device = p->device;
    out->has_quadratic = p->any_w ? 1 : 0;
    return SAIS_OK;
}

sais_status sais_instance_scalars(const sais_problem *p, int32_t index, sais_problem_scalars *out) {
    if (!p || !out) return fail(SAIS_EINVAL, "NULL argument");
    if (index < 0 || index >= p->count) return fail(SAIS_EINVAL, "index %d out of range", index);
    const HostInst &h = p->host[index];
    out->n = h.n;
    out->m = h.m;
    out->n_spins = h.nprime;
    out->words = h.words;
    out->sigma_f = h.sf;
    out->sigma_g = h.sg;
    out->penalty = h.P;
    out->reserved = 0.f;
    out->density = h.d;
    return SAIS_OK;
}

}  // extern "C"

namespace {

sais_status check_sample_params(const sais_problem *p, const sais_sample_params *prm) {
    if (!p || !prm) return fail(SAIS_EINVAL, "NULL problem or params");
    if (prm->chains < 1) return fail(SAIS_EINVAL, "chains = %d: need >= 1", prm->chains);
    if (prm->sweeps < 1) return fail(SAIS_EINVAL, "sweeps = %d: need >= 1", prm->sweeps);
    if (!(prm->beta_max >= 0.0f) || !std::isfinite(prm->beta_max))
        return fail(SAIS_EINVAL, "beta_max must be finite and >= 0");
    if (prm->variant != SAIS_PLAIN && prm->variant != SAIS_BLOCKED && prm->variant != SAIS_AUTO)
        return fail(SAIS_EINVAL, "unknown variant %d", prm->variant);
    if (prm->chains_per_cta != 0 && prm->chains_per_cta != 32 && prm->chains_per_cta != 64 &&
        prm->chains_per_cta != 128)
        return fail(SAIS_EINVAL, "chains_per_cta = %d: need 0, 32, 64 or 128", prm->chains_per_cta);
    if (prm->block_k != 0 && prm->block_k != 16 && prm->block_k != 32 && prm->block_k != 64)
        return fail(SAIS_EINVAL, "block_k = %d: need 0, 16, 32 or 64", prm->block_k);
    if (prm->debug_wait_polls < 0)
        return fail(SAIS_EINVAL, "debug_wait_polls = %d: need >= 0", prm->debug_wait_polls);
    if (prm->variant != SAIS_AUTO && p->count > 65535)
        return fail(SAIS_EUNSUPPORTED,
                    "%d instances: SAIS_PLAIN / SAIS_BLOCKED launch one grid row per instance "
                    "(at most 65535); SAIS_AUTO has no such limit", p->count);
    return SAIS_OK;
}

// Plain sampler CTA size: one warp per CTA by default (shared memory, not threads, bounds how
// many chains an SM holds, so small CTAs pack best), or the caller's choice.
sais_status plain_cpb(const sais_problem *p, int want, int *cpb) {
    const int c = want ? want : 32;
    const size_t need = plain_smem_bytes(p->max_npad_w, p->words, p->any_w, c, p->all_f16);
    if (need > (size_t)kMaxPlainSmem)
        return fail(SAIS_EUNSUPPORTED,
                    "plain sampler: N'=%d needs %zu bytes of shared memory at %d chains per CTA",
                    p->max_spins, need, c);
    *cpb = c;
    return SAIS_OK;
}

// Best-in-run outputs of a sampling launch (all NULL: off).
struct RunOut {
    uint32_t *x = nullptr;
    int64_t *cost = nullptr;
    int32_t *sweep = nullptr;
    int32_t *nfeas = nullptr;
};

// The step-size rule's parameters (sais_update_lambda_rule, sais_solve).
sais_status check_step_rule(double eta_decay, double momentum) {
    if (!std::isfinite(eta_decay) || eta_decay < 0.0)
        return fail(SAIS_EINVAL, "eta_decay = %g: need a finite value >= 0", eta_decay);
    if (!(momentum >= 0.0 && momentum < 1.0))
        return fail(SAIS_EINVAL, "momentum = %g: need 0 <= momentum < 1", momentum);
    return SAIS_OK;
}

// What one sampling launch will run, decided from the handle and the parameters alone, so that
// every size and variant check happens before anything is queued on a stream.
struct SamplePlan {
    int variant = SAIS_PLAIN;   // SAIS_PLAIN, SAIS_BLOCKED or SAIS_AUTO
    bool field = false;         // blocked with per-block field GEMMs on one CTA
    bool stream_w = false;      // rank-k blocked with W tiles streamed instead of resident
    bool hilo = false;          // BF16 hi/lo split of W
    int k = 16;                 // spins per block (blocked)
    int cpb = 0;                // chains per CTA (plain)
};

sais_status plan_sample(const sais_problem *p, const sais_sample_params *prm, SamplePlan *pl) {
    pl->variant = prm->variant;
    if (!p->inst_chains.empty())
        for (int j = 0; j < p->count; ++j)
            if (p->inst_chains[j] > prm->chains)
                return fail(SAIS_EINVAL,
                            "instance %d has %d chains but the chains argument (the row stride) "
                            "is %d", j, p->inst_chains[j], prm->chains);
    if (prm->variant == SAIS_AUTO) {
        for (const auto &g : p->groups)
            if (g.variant == SAIS_PLAIN &&
                plain_smem_bytes(g.max_npad_w, g.words, g.any_w, g.cpb, g.f16) > (size_t)kMaxPlainSmem)
                return fail(SAIS_EUNSUPPORTED,
                            "plain sampler group: padded N'=%d needs %zu bytes of shared memory",
                            g.max_npad_w, plain_smem_bytes(g.max_npad_w, g.words, g.any_w, g.cpb, g.f16));
        return SAIS_OK;
    }
    if (prm->variant == SAIS_PLAIN) return plain_cpb(p, prm->chains_per_cta, &pl->cpb);
    const int k = prm->block_k ? prm->block_k : 16;
    pl->k = k;
    if (!p->all_w)
        return fail(SAIS_EUNSUPPORTED,
                    "blocked sampler: every instance needs a quadratic objective W "
                    "(linear objectives have no dense field to update; use SAIS_PLAIN)");
    if (p->max_m > kMaxBlockedConstraints)
        return fail(SAIS_EUNSUPPORTED,
                    "blocked sampler: m = %d constraints (at most %d; use SAIS_PLAIN)",
                    p->max_m, kMaxBlockedConstraints);
    pl->hilo = p->any_lo;
    // Rank-k update with the fields resident (K = 16; K = 32 with W resident).
    if ((k == 16 || k == 32) && p->max_npad + k <= 512) {
        pl->stream_w = pl->hilo || blocked_smem_bytes(p->max_npad, p->words, k, false, false) >
                                       kMaxSmemPerBlock;
        const size_t smem = blocked_smem_bytes(p->max_npad, p->words, k, pl->stream_w, pl->hilo);
        if ((k == 16 || !pl->stream_w) && smem <= kMaxSmemPerBlock) return SAIS_OK;
    }
    // Block fields from a GEMM over the states (the caller's K, or the default then 16).
    for (int kf : {prm->block_k ? k : field_default_k(p->max_m), k}) {
        if (field_fits(p->max_n16, p->words, p->max_m, true, kf, pl->hilo)) {
            pl->k = kf;
            pl->field = true;
            return SAIS_OK;
        }
    }
    if (k != 16 && p->max_m > 2)
        return fail(SAIS_EUNSUPPORTED,
                    "blocked sampler: block_k = %d takes at most 2 constraints (m = %d)", k,
                    p->max_m);
    if (p->max_n16 > 1024)
        return fail(SAIS_EUNSUPPORTED,
                    "blocked sampler: n = %d items, more than the 1024 its kernels hold (use "
                    "SAIS_PLAIN)", p->max_n);
    return fail(SAIS_EUNSUPPORTED,
                "blocked sampler: block_k = %d with n = %d needs %zu bytes of shared memory (max "
                "%zu)", k, p->max_n, field_smem_bytes(p->max_n16, p->words, k, pl->hilo),
                kMaxSmemPerBlock);
}

sais_status enqueue_sample(sais_problem *p, const sais_sample_params *prm, const float *lambda,
                           const uint32_t *iter_dev, uint32_t *x, int64_t *cost, int64_t *g,
                           uint8_t *feasible, uint32_t *trace, cudaStream_t st,
                           const RunOut &run = RunOut{}) {
    SamplePlan pl;
    sais_status ps = plan_sample(p, prm, &pl);
    if (ps != SAIS_OK) return ps;
    SampleArgs a{};
    a.inst = p->d_inst;
    a.count = p->count;
    a.chains = prm->chains;
    a.sweeps = prm->sweeps;
    a.beta_max = prm->beta_max;
    a.iter = prm->iter;
    a.iter_dev = iter_dev;
    a.seed = prm->seed;
    a.words = p->words;
    a.m_stride = p->m_stride;
    a.lambda = lambda;
    a.x = x;
    a.cost = cost;
    a.g = g;
    a.feasible = feasible;
    a.trace = trace;
    a.run_x = run.x;
    a.run_cost = run.cost;
    a.run_sweep = run.sweep;
    a.run_nfeas = run.nfeas;
    a.status = p->d_status;
    a.inst_chains = p->d_inst_chains;
    const long long polls = (long long)prm->debug_wait_polls;
    cudaError_t e;
    if (pl.variant == SAIS_AUTO) {
        sais_status s = ensure_work(p, prm->chains, st);
        if (s != SAIS_OK) return s;
        if (p->use_ragged) {   // one persistent launch over every instance
            e = launch_ragged(a, p->d_work + p->ragged_off, (int32_t)p->ragged_n,
                              p->d_work + p->head_off,
                              reinterpret_cast<unsigned long long *>(p->d_work + p->stats_off),
                              p->max_n16, p->words, p->any_lo,
                              p->d_status, polls, p->sms, st);
            if (e != cudaSuccess)
                return fail(SAIS_ECUDA, "sampler launch (persistent): %s", cudaGetErrorString(e));
            return SAIS_OK;
        }
        if (p->groups.size() == 1) {
            e = launch_group(p, p->groups[0], a, polls, st);
            if (e != cudaSuccess)
                return fail(SAIS_ECUDA, "sampler launch (group): %s", cudaGetErrorString(e));
            return SAIS_OK;
        }
        e = cudaEventRecord(p->fork, st);
        std::vector<char> used(p->side.size(), 0);
        for (size_t gi = 0; e == cudaSuccess && gi < p->groups.size(); ++gi) {
            const auto &g = p->groups[gi];
            if (g.nwork == 0) continue;
            const size_t si = gi + 1;
            if (!used[si]) e = cudaStreamWaitEvent(p->side[si], p->fork, 0);
            used[si] = 1;
            if (e == cudaSuccess) e = launch_group(p, g, a, polls, p->side[si]);
        }
        for (size_t si = 0; e == cudaSuccess && si < p->side.size(); ++si) {
            if (!used[si]) continue;
            e = cudaEventRecord(p->join[si], p->side[si]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->join[si], 0);
        }
        if (e != cudaSuccess)
            return fail(SAIS_ECUDA, "sampler launch (groups): %s", cudaGetErrorString(e));
        return SAIS_OK;
    }
    if (pl.variant == SAIS_BLOCKED && pl.field)
        e = launch_field_sampler(a, p->max_m, p->max_n16, p->words, pl.k, pl.hilo, p->d_status,
                                 polls, st);
    else if (pl.variant == SAIS_BLOCKED)
        e = launch_blocked_sampler(a, p->max_m, p->max_npad, p->words, pl.k, pl.stream_w, pl.hilo,
                                   p->d_status, polls, st);
    else
        e = launch_plain_sampler(a, p->max_m, p->max_npad_w, p->words, pl.cpb, st, p->all_f16);
    if (e != cudaSuccess) return fail(SAIS_ECUDA, "sampler launch: %s", cudaGetErrorString(e));
    return SAIS_OK;
}

}  // namespace

extern "C" {

sais_status sais_sample(sais_problem *p, const sais_sample_params *prm, const float *lambda,
                        uint32_t *x, int64_t *cost, int64_t *g, uint8_t *feasible, void *stream) {
    NvtxRange nvtx_range("sais_sample");
    sais_status s = check_sample_params(p, prm);
    if (s != SAIS_OK) return s;
    if (!lambda || !x || !cost || !g) return fail(SAIS_EINVAL, "NULL device buffer");
    DeviceGuard dg(p->device);
    return enqueue_sample(p, prm, lambda, nullptr, x, cost, g, feasible, nullptr,
                          static_cast<cudaStream_t>(stream));
}

sais_status sais_sample_trace(sais_problem *p, const sais_sample_params *prm, const float *lambda,
                              uint32_t *x, int64_t *cost, int64_t *g, uint8_t *feasible,
                              uint32_t *trace, void *stream) {
    NvtxRange nvtx_range("sais_sample_trace");
    sais_status s = check_sample_params(p, prm);
    if (s != SAIS_OK) return s;
    if (!lambda || !x || !cost || !g || !trace) return fail(SAIS_EINVAL, "NULL device buffer");
    DeviceGuard dg(p->device);
    return enqueue_sample(p, prm, lambda, nullptr, x, cost, g, feasible, trace,
                          static_cast<cudaStream_t>(stream));
}

sais_status sais_sample_run_best(sais_problem *p, const sais_sample_params *prm,
                                 const float *lambda, uint32_t *x, int64_t *cost, int64_t *g,
                                 uint8_t *feasible, uint32_t *run_x, int64_t *run_cost,
                                 int32_t *run_sweep, int32_t *run_nfeas, void *stream) {
    NvtxRange nvtx_range("sais_sample_run_best");
    sais_status s = check_sample_params(p, prm);
    if (s != SAIS_OK) return s;
    if (!lambda || !x || !cost || !g || !run_x || !run_cost)
        return fail(SAIS_EINVAL, "NULL device buffer");
    DeviceGuard dg(p->device);
    RunOut run;
    run.x = run_x;
    run.cost = run_cost;
    run.sweep = run_sweep;
    run.nfeas = run_nfeas;
    return enqueue_sample(p, prm, lambda, nullptr, x, cost, g, feasible, nullptr,
                          static_cast<cudaStream_t>(stream), run);
}

sais_status sais_sample_plan(const sais_problem *p, const sais_sample_params *prm,
                             sais_plan *out) {
    if (!out) return fail(SAIS_EINVAL, "out is NULL");
    sais_status s = check_sample_params(p, prm);
    if (s != SAIS_OK) return s;
    SamplePlan pl;
    s = plan_sample(p, prm, &pl);
    if (s != SAIS_OK) return s;
    *out = sais_plan{};
    if (pl.variant == SAIS_AUTO) {
        out->kernel = p->use_ragged ? SAIS_KERNEL_PERSISTENT : SAIS_KERNEL_GROUPS;
        out->hilo = p->any_lo ? 1 : 0;
    } else if (pl.variant == SAIS_PLAIN) {
        out->kernel = SAIS_KERNEL_PLAIN;
        out->chains_per_cta = pl.cpb;
    } else {
        out->kernel = pl.field ? SAIS_KERNEL_BLOCK_FIELD
                               : (pl.stream_w ? SAIS_KERNEL_RANKK_STREAMED
                                              : SAIS_KERNEL_RANKK_RESIDENT);
        out->block_k = pl.k;
        out->chains_per_cta = 128;
        out->hilo = pl.hilo ? 1 : 0;
    }
    return SAIS_OK;
}

sais_status sais_set_auto_mode(sais_problem *p, int32_t mode) {
    if (!p) return fail(SAIS_EINVAL, "NULL problem");
    if (mode != SAIS_AUTO_PERSISTENT && mode != SAIS_AUTO_GROUPS)
        return fail(SAIS_EINVAL, "unknown SAIS_AUTO mode %d", mode);
    p->use_ragged = mode == SAIS_AUTO_PERSISTENT && p->ragged_ok;
    return SAIS_OK;
}

sais_status sais_persistent_stats(sais_problem *p, uint64_t *out, int32_t cap, int32_t *ctas,
                                  void *stream) {
    if (!p || !out || !ctas || cap < 0) return fail(SAIS_EINVAL, "NULL argument or cap < 0");
    if (!p->ragged_ok || !p->work_valid || p->ragged_ctas == 0)
        return fail(SAIS_EINVAL, "no persistent launch prepared for this problem");
    DeviceGuard dg(p->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    *ctas = p->ragged_ctas;
    const size_t n = (size_t)std::min(cap, p->ragged_ctas) * 4;
    SAIS_CUDA(cudaMemcpyAsync(out, p->d_work + p->stats_off, n * sizeof(uint64_t),
                              cudaMemcpyDeviceToHost, st));
    SAIS_CUDA(cudaStreamSynchronize(st));
    return SAIS_OK;
}

sais_status sais_debug_check_selftest(sais_problem *p, void *stream) {
    if (!p) return fail(SAIS_EINVAL, "NULL problem");
    if (!debug_checks_built())
        return fail(SAIS_EUNSUPPORTED, "device-side checks are compiled in debug builds only "
                                       "(SAIS_DEBUG=1)");
    DeviceGuard dg(p->device);
    const cudaError_t e = launch_dcheck_selftest(p->d_status, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(SAIS_ECUDA, "check self-test: %s", cudaGetErrorString(e));
    return SAIS_OK;
}

sais_status sais_synchronize(sais_problem *p, void *stream) {
    if (!p) return fail(SAIS_EINVAL, "NULL problem");
    DeviceGuard dg(p->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SAIS_CUDA(cudaStreamSynchronize(st));
    int32_t v[2] = {0, 0};   // the status, and the source line of a failed debug check
    SAIS_CUDA(cudaMemcpy(v, p->d_status, 8, cudaMemcpyDeviceToHost));
    if (v[0] != SAIS_OK) {
        SAIS_CUDA(cudaMemset(p->d_status, 0, 8));
        if (v[0] == SAIS_EBOUNDS)
            return fail(SAIS_EBOUNDS, "a kernel on this problem reported: %s (check at line %d)",
                        sais_status_string(SAIS_EBOUNDS), v[1]);
        return fail((sais_status)v[0], "a kernel on this problem reported: %s",
                    sais_status_string((sais_status)v[0]));
    }
    return SAIS_OK;
}

sais_status sais_update_lambda(sais_problem *p, const int64_t *g, int32_t chains, double eta,
                               int32_t project_nonneg, float *lambda, void *stream) {
    NvtxRange nvtx_range("sais_update_lambda");
    if (!p || !g || !lambda) return fail(SAIS_EINVAL, "NULL argument");
    if (chains < 1) return fail(SAIS_EINVAL, "chains = %d: need >= 1", chains);
    if (!std::isfinite(eta)) return fail(SAIS_EINVAL, "eta must be finite");
    DeviceGuard dg(p->device);
    PostArgs a{};
    a.inst = p->d_inst;
    a.count = p->count;
    a.chains = chains;
    a.words = p->words;
    a.m_stride = p->m_stride;
    a.eta = eta;
    a.project = project_nonneg ? 1 : 0;
    a.track_best = 0;
    a.do_lambda = 1;
    a.inst_chains = p->d_inst_chains;
    a.g = g;
    a.lambda = lambda;
    cudaError_t e = launch_post(a, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(SAIS_ECUDA, "multiplier update launch: %s", cudaGetErrorString(e));
    return SAIS_OK;
}

sais_status sais_update_lambda_rule(sais_problem *p, const int64_t *g, int32_t chains,
                                    double eta, int32_t project_nonneg, uint32_t iter,
                                    double eta_decay, int32_t eta_sqrt, double momentum,
                                    double *avg, float *lambda, void *stream) {
    NvtxRange nvtx_range("sais_update_lambda_rule");
    if (!p || !g || !lambda) return fail(SAIS_EINVAL, "NULL argument");
    if (chains < 1) return fail(SAIS_EINVAL, "chains = %d: need >= 1", chains);
    if (!std::isfinite(eta)) return fail(SAIS_EINVAL, "eta must be finite");
    sais_status s = check_step_rule(eta_decay, momentum);
    if (s != SAIS_OK) return s;
    if (momentum != 0.0 && !avg) return fail(SAIS_EINVAL, "avg is NULL with momentum != 0");
    DeviceGuard dg(p->device);
    PostArgs a{};
    a.inst = p->d_inst;
    a.count = p->count;
    a.chains = chains;
    a.words = p->words;
    a.m_stride = p->m_stride;
    a.eta = eta;
    a.project = project_nonneg ? 1 : 0;
    a.eta_decay = eta_decay;
    a.eta_sqrt = eta_sqrt ? 1 : 0;
    a.momentum = momentum;
    a.avg = avg;
    a.iter = iter;
    a.track_best = 0;
    a.do_lambda = 1;
    a.inst_chains = p->d_inst_chains;
    a.g = g;
    a.lambda = lambda;
    cudaError_t e = launch_post(a, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(SAIS_ECUDA, "multiplier update launch: %s", cudaGetErrorString(e));
    return SAIS_OK;
}

sais_status sais_track_best(sais_problem *p, const uint32_t *x, const int64_t *cost,
                            const uint8_t *feasible, int32_t chains, uint32_t iter,
                            int64_t *best_cost, uint32_t *best_x, int32_t *best_iter,
                            int32_t *best_chain, int64_t *feasible_count, void *stream) {
    NvtxRange nvtx_range("sais_track_best");
    if (!p || !x || !cost || !best_cost || !best_x || !best_iter || !best_chain || !feasible_count)
        return fail(SAIS_EINVAL, "NULL argument");
    if (chains < 1) return fail(SAIS_EINVAL, "chains = %d: need >= 1", chains);
    DeviceGuard dg(p->device);
    PostArgs a{};
    a.inst = p->d_inst;
    a.count = p->count;
    a.chains = chains;
    a.words = p->words;
    a.m_stride = p->m_stride;
    a.track_best = 1;
    a.do_lambda = 0;
    a.inst_chains = p->d_inst_chains;
    a.x = x;
    a.cost = cost;
    a.feasible = feasible;
    a.iter = iter;
    a.best_cost = best_cost;
    a.best_x = best_x;
    a.best_iter = best_iter;
    a.best_chain = best_chain;
    a.feasible_count = feasible_count;
    cudaError_t e = launch_post(a, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(SAIS_ECUDA, "best-tracking launch: %s", cudaGetErrorString(e));
    return SAIS_OK;
}

sais_status sais_solve(sais_problem *p, const sais_solve_params *prm, sais_solve_result *res,
                       void *stream) {
    NvtxRange nvtx_range("sais_solve");
    if (!p || !prm || !res) return fail(SAIS_EINVAL, "NULL argument");
    if (prm->iters < 1) return fail(SAIS_EINVAL, "iters = %d: need >= 1", prm->iters);
    if (!std::isfinite(prm->eta)) return fail(SAIS_EINVAL, "eta must be finite");
    {
        sais_status r = check_step_rule(prm->eta_decay, prm->momentum);
        if (r != SAIS_OK) return r;
    }
    sais_sample_params sp{};
    sp.chains = prm->chains;
    sp.sweeps = prm->sweeps;
    sp.beta_max = prm->beta_max;
    sp.iter = prm->iter0;
    sp.seed = prm->seed;
    sp.variant = prm->variant;
    sp.block_k = prm->block_k;
    sp.chains_per_cta = prm->chains_per_cta;
    sais_status s = check_sample_params(p, &sp);
    if (s != SAIS_OK) return s;
    DeviceGuard dg(p->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    const int count = p->count, C = prm->chains, K = prm->iters;
    const size_t nch = (size_t)count * C;
    // Device scratch owned by this call.
    size_t sz_lam = (size_t)count * p->m_stride * 4, sz_x = nch * p->words * 4, sz_cost = nch * 8,
           sz_g = nch * p->m_stride * 8, sz_feas = nch, sz_bc = (size_t)count * 8,
           sz_bx = (size_t)count * p->words * 4, sz_bi = (size_t)count * 4,
           sz_fc = (size_t)count * 8, sz_tr = (size_t)K * count * p->m_stride * 4;
    const bool rb = prm->run_best != 0;
    const size_t sz_avg = prm->momentum != 0.0 ? (size_t)count * p->m_stride * 8 : 0;
    size_t offs[15], cur = 0;
    const size_t sizes[15] = {sz_lam, sz_x, sz_cost, sz_g, sz_feas, sz_bc, sz_bx, sz_bi, sz_bi,
                              sz_fc, sz_tr, 4, rb ? sz_x : 0, rb ? sz_cost : 0, sz_avg};
    for (int i = 0; i < 15; ++i) {
        offs[i] = cur;
        cur = align_up(cur + sizes[i], 256);
    }
    unsigned char *scr = nullptr;
    SAIS_CUDA(dev_alloc(reinterpret_cast<void **>(&scr), cur));
    struct Free {   // on every return: the call's work done, then the scratch released
        unsigned char *q;
        cudaStream_t s;
        ~Free() {
            cudaStreamSynchronize(s);
            dev_free(q);
        }
    } free_scr{scr, st};
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
    RunOut run;   // best-in-run: the kept sample of a chain is its best feasible sweep end
    if (rb) {
        run.x = reinterpret_cast<uint32_t *>(scr + offs[12]);
        run.cost = reinterpret_cast<int64_t *>(scr + offs[13]);
    }

    std::vector<int64_t> h_bc(count, std::numeric_limits<int64_t>::max());
    std::vector<int32_t> h_m1(count, -1);
    SAIS_CUDA(cudaMemsetAsync(scr, 0, cur, st));
    if (prm->lambda0)
        SAIS_CUDA(cudaMemcpyAsync(d_lam, prm->lambda0, sz_lam, cudaMemcpyHostToDevice, st));
    SAIS_CUDA(cudaMemcpyAsync(d_bc, h_bc.data(), sz_bc, cudaMemcpyHostToDevice, st));
    SAIS_CUDA(cudaMemcpyAsync(d_bi, h_m1.data(), sz_bi, cudaMemcpyHostToDevice, st));
    SAIS_CUDA(cudaMemcpyAsync(d_bch, h_m1.data(), sz_bi, cudaMemcpyHostToDevice, st));
    SAIS_CUDA(cudaMemcpyAsync(d_iter, &prm->iter0, 4, cudaMemcpyHostToDevice, st));

    PostArgs pa{};
    pa.inst = p->d_inst;
    pa.count = count;
    pa.chains = C;
    pa.words = p->words;
    pa.m_stride = p->m_stride;
    pa.eta = prm->eta;
    pa.project = prm->project_nonneg ? 1 : 0;
    pa.eta_decay = prm->eta_decay;
    pa.eta_sqrt = prm->eta_sqrt ? 1 : 0;
    pa.momentum = prm->momentum;
    pa.avg = sz_avg ? reinterpret_cast<double *>(scr + offs[14]) : nullptr;   // zeroed below
    pa.track_best = 1;
    pa.do_lambda = 1;
    pa.inst_chains = p->d_inst_chains;
    pa.x = rb ? run.x : d_x;
    pa.cost = rb ? run.cost : d_cost;
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

    auto one_iteration = [&]() -> sais_status {
        sais_status r = enqueue_sample(p, &sp, d_lam, d_iter, d_x, d_cost, d_g, d_feas, nullptr, st,
                                       run);
        if (r != SAIS_OK) return r;
        cudaError_t e = launch_post(pa, st);
        if (e == cudaSuccess) e = launch_advance_iter(d_iter, st);
        if (e != cudaSuccess) return fail(SAIS_ECUDA, "post launch: %s", cudaGetErrorString(e));
        return SAIS_OK;
    };

    cudaEvent_t ev0, ev1;
    SAIS_CUDA(cudaEventCreate(&ev0));
    SAIS_CUDA(cudaEventCreate(&ev1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } evs{ev0, ev1};
    cudaGraphExec_t exec = nullptr;
    if (prm->variant == SAIS_AUTO) {
        sais_status r = ensure_work(p, C, st);
        if (r != SAIS_OK) return r;
    }
    if (prm->use_graph) {
        cudaStream_t cap = st;
        bool own = false;
        if (cap == nullptr) {  // the legacy stream cannot be captured
            SAIS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            own = true;
        }
        cudaStream_t saved = st;
        st = cap;
        cudaGraph_t graph = nullptr;
        SAIS_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
        sais_status r = one_iteration();
        cudaError_t e = cudaStreamEndCapture(cap, &graph);
        if (r != SAIS_OK) {
            if (graph) cudaGraphDestroy(graph);
            if (own) cudaStreamDestroy(cap);
            return r;
        }
        if (e != cudaSuccess) {
            if (own) cudaStreamDestroy(cap);
            return fail(SAIS_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (own) cudaStreamDestroy(cap);
        st = saved;
        if (e != cudaSuccess) return fail(SAIS_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    SAIS_CUDA(cudaEventRecord(ev0, st));
    for (int k = 0; k < K; ++k) {
        NvtxRange nvtx_iter("sais_solve iteration");
        if (exec) {
            cudaError_t e = cudaGraphLaunch(exec, st);
            if (e != cudaSuccess) {
                cudaGraphExecDestroy(exec);
                return fail(SAIS_ECUDA, "graph launch: %s", cudaGetErrorString(e));
            }
        } else {
            sais_status r = one_iteration();
            if (r != SAIS_OK) return r;
        }
    }
    SAIS_CUDA(cudaEventRecord(ev1, st));
    if (exec) cudaGraphExecDestroy(exec);

    if (res->best_cost) SAIS_CUDA(cudaMemcpyAsync(res->best_cost, d_bc, sz_bc, cudaMemcpyDeviceToHost, st));
    if (res->best_x) SAIS_CUDA(cudaMemcpyAsync(res->best_x, d_bx, sz_bx, cudaMemcpyDeviceToHost, st));
    if (res->best_iter) SAIS_CUDA(cudaMemcpyAsync(res->best_iter, d_bi, sz_bi, cudaMemcpyDeviceToHost, st));
    if (res->best_chain) SAIS_CUDA(cudaMemcpyAsync(res->best_chain, d_bch, sz_bi, cudaMemcpyDeviceToHost, st));
    if (res->feasible_count) SAIS_CUDA(cudaMemcpyAsync(res->feasible_count, d_fc, sz_fc, cudaMemcpyDeviceToHost, st));
    if (res->lambda_final) SAIS_CUDA(cudaMemcpyAsync(res->lambda_final, d_lam, sz_lam, cudaMemcpyDeviceToHost, st));
    if (res->lambda_trace) SAIS_CUDA(cudaMemcpyAsync(res->lambda_trace, d_tr, sz_tr, cudaMemcpyDeviceToHost, st));
    SAIS_CUDA(cudaStreamSynchronize(st));
    {
        int32_t v = 0;
        SAIS_CUDA(cudaMemcpy(&v, p->d_status, 4, cudaMemcpyDeviceToHost));
        if (v != SAIS_OK) {
            SAIS_CUDA(cudaMemset(p->d_status, 0, 4));
            return fail((sais_status)v, "a sampler kernel reported: %s",
                        sais_status_string((sais_status)v));
        }
    }
    float ms = 0.f;
    SAIS_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
    res->elapsed_ms = ms;
    int64_t upd = 0;
    for (int j = 0; j < count; ++j)
        upd += (int64_t)p->host[j].nprime *
               (p->inst_chains.empty() ? (int64_t)C : (int64_t)p->inst_chains[j]);
    res->spin_updates = upd * (int64_t)prm->sweeps * K;
    return SAIS_OK;
}

}  // extern "C"

extern "C" {

sais_status sais_set_instance_chains(sais_problem *p, const int32_t *counts) {
    if (!p) return fail(SAIS_EINVAL, "NULL problem");
    DeviceGuard dg(p->device);
    if (!counts) {
        p->inst_chains.clear();
        if (p->d_inst_chains) {
            cudaDeviceSynchronize();   // queued launches may still read the counts
            dev_free(p->d_inst_chains);
        }
        p->d_inst_chains = nullptr;
        p->work_valid = false;
        return SAIS_OK;
    }
    for (int j = 0; j < p->count; ++j)
        if (counts[j] < 1) return fail(SAIS_EINVAL, "counts[%d] = %d: need >= 1", j, counts[j]);
    if (!p->d_inst_chains) {
        cudaError_t e = dev_alloc(reinterpret_cast<void **>(&p->d_inst_chains),
                                  (size_t)p->count * 4);
        if (e != cudaSuccess) return fail(SAIS_ENOMEM, "chain counts: %s", cudaGetErrorString(e));
    }
    cudaError_t e = cudaMemcpy(p->d_inst_chains, counts, (size_t)p->count * 4,
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(SAIS_ECUDA, "chain counts copy: %s", cudaGetErrorString(e));
    p->inst_chains.assign(counts, counts + p->count);
    p->work_valid = false;
    return SAIS_OK;
}

sais_status sais_autotune(sais_problem *p, int32_t chains, int32_t sweeps, sais_tuning *out,
                          void *stream) {
    NvtxRange nvtx_range("sais_autotune");
    if (!p || !out) return fail(SAIS_EINVAL, "NULL argument");
    if (chains < 1 || sweeps < 1) return fail(SAIS_EINVAL, "need chains >= 1 and sweeps >= 1");
    DeviceGuard dg(p->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t nch = (size_t)p->count * chains;
    const size_t sz[5] = {nch * p->words * 4, nch * 8, nch * p->m_stride * 8, nch,
                          (size_t)p->count * p->m_stride * 4};
    size_t off[5], cur = 0;
    for (int i = 0; i < 5; ++i) {
        off[i] = cur;
        cur = align_up(cur + sz[i], 256);
    }
    unsigned char *buf = nullptr;
    SAIS_CUDA(dev_alloc(reinterpret_cast<void **>(&buf), cur));
    struct Free {   // on every return: the timing launches done, then the buffer released
        unsigned char *q;
        cudaStream_t s;
        ~Free() {
            cudaStreamSynchronize(s);
            dev_free(q);
        }
    } fr{buf, st};
    SAIS_CUDA(cudaMemsetAsync(buf, 0, cur, st));
    cudaEvent_t e0, e1;
    SAIS_CUDA(cudaEventCreate(&e0));
    SAIS_CUDA(cudaEventCreate(&e1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } evs{e0, e1};
    sais_sample_params sp{};
    sp.chains = chains;
    sp.sweeps = sweeps;
    sp.beta_max = 10.0f;
    sp.seed = 1;
    SampleArgs a{};
    a.inst = p->d_inst;
    a.count = p->count;
    a.chains = chains;
    a.sweeps = sweeps;
    a.beta_max = sp.beta_max;
    a.seed = sp.seed;
    a.words = p->words;
    a.m_stride = p->m_stride;
    a.lambda = reinterpret_cast<const float *>(buf + off[4]);
    a.x = reinterpret_cast<uint32_t *>(buf + off[0]);
    a.cost = reinterpret_cast<int64_t *>(buf + off[1]);
    a.g = reinterpret_cast<int64_t *>(buf + off[2]);
    a.feasible = buf + off[3];
    a.status = p->d_status;
    a.inst_chains = p->d_inst_chains;
    std::memset(out, 0, sizeof *out);
    for (size_t gi = 0; gi < p->groups.size(); ++gi) {
        auto &g = p->groups[gi];
        struct Cand {
            int variant, k, cpb;
        };
        std::vector<Cand> cands;
        if (g.blocked_ok && g.field) {
            for (int k : {16, 32, 64})
                if (field_fits(g.max_n16, g.words, g.max_m, true, k, g.hilo))
                    cands.push_back({SAIS_BLOCKED, k, g.cpb});
        } else if (g.blocked_ok) {
            cands.push_back({SAIS_BLOCKED, 16, g.cpb});
            if (!g.stream_w &&
                blocked_smem_bytes(g.max_npad, g.words, 32, false, false) <= kMaxSmemPerBlock &&
                g.max_npad + 32 <= 512)
                cands.push_back({SAIS_BLOCKED, 32, g.cpb});
        }
        for (int cpb : {32, 64, 128})
            if (plain_smem_bytes(g.max_npad_w, g.words, g.any_w, cpb, g.f16) <= (size_t)kMaxPlainSmem)
                cands.push_back({SAIS_PLAIN, g.block_k, cpb});
        double best = 1e300;
        Cand pick = cands.front();
        for (const Cand &c : cands) {
            g.variant = c.variant;
            g.block_k = c.k;
            g.cpb = c.cpb;
            p->work_valid = false;
            sais_status r = ensure_work(p, chains, st);
            if (r != SAIS_OK) return r;
            cudaError_t e = launch_group(p, g, a, 0, st);   // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = launch_group(p, g, a, 0, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) return fail(SAIS_ECUDA, "autotune launch: %s", cudaGetErrorString(e));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                pick = c;
            }
        }
        g.variant = pick.variant;
        g.block_k = pick.k;
        g.cpb = pick.cpb;
        g.tuned_ms = best;
        if (gi < 16) {
            out->group_variant[gi] = g.variant;
            out->group_block_k[gi] = g.variant == SAIS_BLOCKED ? g.block_k : 0;
            out->group_chains_per_cta[gi] = g.variant == SAIS_PLAIN ? g.cpb : 128;
            out->group_size[gi] = (int32_t)g.members.size();
            out->group_ms[gi] = best;
            long long upd = 0;
            for (int j : g.members)
                upd += (long long)p->host[j].nprime *
                       (p->inst_chains.empty() ? chains : p->inst_chains[j]);
            out->group_spin_updates[gi] = (int64_t)upd * sweeps;
        }
        (g.variant == SAIS_BLOCKED ? out->blocked_instances : out->plain_instances) +=
            (int32_t)g.members.size();
    }
    out->groups = (int32_t)p->groups.size();
    // The two ways SAIS_AUTO can run the batch: the concurrent group launches (with the
    // choices above) and, when the batch fits it, one persistent launch; the faster is kept.
    {
        sais_sample_params sa = sp;
        sa.variant = SAIS_AUTO;
        auto time_auto = [&](bool ragged, double *ms) -> sais_status {
            p->use_ragged = ragged;
            p->work_valid = false;
            for (int rep = 0; rep < 2; ++rep) {   // warm-up, then the timed launch
                if (rep == 1) SAIS_CUDA(cudaEventRecord(e0, st));
                sais_status r = enqueue_sample(p, &sa, a.lambda, nullptr, a.x, a.cost, a.g,
                                               a.feasible, nullptr, st);
                if (r != SAIS_OK) return r;
            }
            SAIS_CUDA(cudaEventRecord(e1, st));
            SAIS_CUDA(cudaEventSynchronize(e1));
            float f = 0.f;
            cudaEventElapsedTime(&f, e0, e1);
            *ms = f;
            return SAIS_OK;
        };
        double gms = 0.0, rms = 0.0;
        sais_status r = time_auto(false, &gms);
        if (r != SAIS_OK) return r;
        if (p->ragged_ok) {
            r = time_auto(true, &rms);
            if (r != SAIS_OK) return r;
        }
        p->use_ragged = p->ragged_ok && rms < gms;
        out->persistent_ok = p->ragged_ok ? 1 : 0;
        out->persistent = p->use_ragged ? 1 : 0;
        out->persistent_ms = rms;
        out->groups_ms = gms;
    }
    p->work_valid = false;
    int32_t v = 0;
    SAIS_CUDA(cudaMemcpy(&v, p->d_status, 4, cudaMemcpyDeviceToHost));
    if (v != SAIS_OK) {
        cudaMemset(p->d_status, 0, 4);
        return fail((sais_status)v, "a sampler kernel reported: %s", sais_status_string((sais_status)v));
    }
    return SAIS_OK;
}

}  // extern "C"

extern "C" {

sais_status sais_constraint_features(const sais_problem *p, float *out, int32_t capacity_rows,
                                     int32_t *rows) {
    if (!p || !out || !rows) return fail(SAIS_EINVAL, "NULL argument");
    *rows = p->feat_rows;
    if (capacity_rows < p->feat_rows)
        return fail(SAIS_EINVAL, "capacity of %d rows, %d needed", capacity_rows, p->feat_rows);
    size_t r = 0;
    for (const HostInst &h : p->host)
        for (int32_t k = 0; k < h.m; ++k, ++r)
            std::memcpy(out + r * 8, &h.feat[(size_t)k * 8], 8 * 4);
    return SAIS_OK;
}

sais_status sais_warm_start(sais_problem *p, const sais_mlp *m, float *lambda, void *stream) {
    NvtxRange nvtx_range("sais_warm_start");
    if (!p || !m || !lambda) return fail(SAIS_EINVAL, "NULL argument");
    DeviceGuard dg(p->device);
    return mlp_warm_start_launch(m, p->d_feat, p->d_feat_dst, p->feat_rows, lambda, p->device,
                                 static_cast<cudaStream_t>(stream));
}

}  // extern "C"

// ---- internal accessors for entry points in other translation units ----------------------

namespace sais {

sais_status problem_view(const sais_problem *p, ProblemView *out) {
    if (!p || !out) return fail(SAIS_EINVAL, "NULL argument");
    out->device = p->device;
    out->count = p->count;
    out->words = p->words;
    out->m_stride = p->m_stride;
    out->d_inst = p->d_inst;
    out->d_status = p->d_status;
    out->d_inst_chains = p->d_inst_chains;
    long long tot = 0, totc = 0;
    for (int j = 0; j < p->count; ++j) {
        tot += p->host[j].nprime;
        totc += (long long)p->host[j].nprime * (p->inst_chains.empty() ? 0 : p->inst_chains[j]);
    }
    out->spins_total = tot;
    out->spin_chains_total = totc;
    return SAIS_OK;
}

sais_status enqueue_sample_internal(sais_problem *p, const sais_sample_params *prm,
                                   const float *lambda, const uint32_t *iter_dev, uint32_t *x,
                                   int64_t *cost, int64_t *g, uint8_t *feasible,
                                   uint32_t *run_x, int64_t *run_cost, cudaStream_t stream) {
    RunOut run;
    run.x = run_x;
    run.cost = run_cost;
    return enqueue_sample(p, prm, lambda, iter_dev, x, cost, g, feasible, nullptr, stream, run);
}

sais_status check_sample_params_internal(const sais_problem *p, const sais_sample_params *prm) {
    sais_status s = check_sample_params(p, prm);
    if (s != SAIS_OK) return s;
    SamplePlan pl;
    return plan_sample(p, prm, &pl);
}

sais_status check_step_rule_internal(double eta_decay, double momentum) {
    return check_step_rule(eta_decay, momentum);
}

namespace {

struct DevAllocator {
    sais_device_alloc_fn alloc = nullptr;   // NULL: cudaMalloc / cudaFree
    sais_device_free_fn free = nullptr;
    void *ctx = nullptr;
};
struct DevBlock {
    DevAllocator by;
    size_t bytes;
    int device;
};
std::mutex g_alloc_lock;
DevAllocator g_allocator;
std::unordered_map<void *, DevBlock> g_blocks;   // blocks of the caller's allocators

}  // namespace

cudaError_t dev_alloc(void **ptr, size_t bytes) {
    *ptr = nullptr;
    DevAllocator a;
    {
        std::lock_guard<std::mutex> lock(g_alloc_lock);
        a = g_allocator;
    }
    if (!a.alloc) return cudaMalloc(ptr, bytes);
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    void *p = a.alloc(bytes, device, a.ctx);
    if (!p) return cudaErrorMemoryAllocation;
    if (reinterpret_cast<uintptr_t>(p) % 256 != 0) {
        a.free(p, bytes, device, a.ctx);
        return cudaErrorMemoryAllocation;
    }
    {
        std::lock_guard<std::mutex> lock(g_alloc_lock);
        g_blocks[p] = DevBlock{a, bytes, device};
    }
    *ptr = p;
    return cudaSuccess;
}

void dev_free(void *ptr) {
    if (!ptr) return;
    DevBlock b{};
    bool mine = false;
    {
        std::lock_guard<std::mutex> lock(g_alloc_lock);
        auto it = g_blocks.find(ptr);
        if (it != g_blocks.end()) {
            b = it->second;
            g_blocks.erase(it);
            mine = true;
        }
    }
    if (mine)
        b.by.free(ptr, b.bytes, b.device, b.by.ctx);
    else
        cudaFree(ptr);
}

sais_status set_error(sais_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

}  // namespace sais

extern "C" sais_status sais_set_device_allocator(sais_device_alloc_fn alloc_fn,
                                                 sais_device_free_fn free_fn, void *ctx) {
    using namespace sais;
    if ((alloc_fn == nullptr) != (free_fn == nullptr))
        return set_error(SAIS_EINVAL, "give both an alloc and a free function, or neither");
    std::lock_guard<std::mutex> lock(g_alloc_lock);
    g_allocator = DevAllocator{alloc_fn, free_fn, alloc_fn ? ctx : nullptr};
    return SAIS_OK;
}
