// C ABI of include/projection.h: argument checks, the host-side parameter
// choice of Section 5, and the orchestration of the whole path
// (Algorithm 2 + Section 5.1) on one stream.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "em_batch.cuh"

namespace proj {

static thread_local char g_err[512];

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

// One stream-ordered memory pool per device, owned by the library, that keeps
// freed blocks for reuse (release threshold = unlimited): scratch allocated and
// freed on every call is then recycled instead of being unmapped and mapped
// again at each synchronisation.  The process's default pool is not touched.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];

static int library_pool(cudaMemPool_t *out) {
    int dev = 0;
    PROJ_CUDA_TRY(cudaGetDevice(&dev));
    PROJ_REQUIRE(dev >= 0 && dev < 64, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        PROJ_CUDA_TRY(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = ~0ull;
        PROJ_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return PROJ_OK;
}

int DevBuf::alloc(size_t bytes, cudaStream_t st) {
    release();
    st_ = st;
    bytes_ = bytes;
    if (bytes == 0) return PROJ_OK;
    cudaMemPool_t pool;
    PROJ_TRY(library_pool(&pool));
    cudaError_t e = cudaMallocFromPoolAsync(&ptr_, bytes, pool, st);
    if (e != cudaSuccess) {
        ptr_ = nullptr;
        bytes_ = 0;
        set_error("cudaMallocAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
        return PROJ_ENOMEM;
    }
    return PROJ_OK;
}

void DevBuf::release() {
    if (ptr_) cudaFreeAsync(ptr_, st_);
    ptr_ = nullptr;
    bytes_ = 0;
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

int make_layout(const int64_t *seq_off, int t, int l, cudaStream_t st, Layout &L) {
    PROJ_REQUIRE(seq_off != nullptr, "seq_off must not be NULL");
    PROJ_REQUIRE(t >= 1, "need t >= 1, got %d", t);
    PROJ_REQUIRE(l >= 1 && l <= 32, "need 1 <= l <= 32, got %d", l);
    PROJ_REQUIRE(seq_off[0] == 0, "seq_off[0] must be 0");
    L.t = t;
    L.l = l;
    L.seq_off.resize(t + 1);
    L.lmer_off.resize(t + 1);
    L.lmer_off[0] = 0;
    L.seq_off[0] = 0;
    int64_t x = 0;
    int max_ns = 0;
    for (int i = 0; i < t; ++i) {
        const int64_t n = seq_off[i + 1] - seq_off[i];
        PROJ_REQUIRE(n >= l, "sequence %d has length %lld < l = %d", i, (long long)n, l);
        PROJ_REQUIRE(seq_off[i + 1] < ((int64_t)1 << 31), "input longer than 2^31 - 1 bases");
        x += n - l + 1;
        max_ns = (int)std::max<int64_t>(max_ns, n - l + 1);
        L.seq_off[i + 1] = (int32_t)seq_off[i + 1];
        L.lmer_off[i + 1] = (int32_t)x;
    }
    L.total = seq_off[t];
    L.x = x;
    L.max_ns = max_ns;
    L.nwords = (L.total + 15) / 16;
    PROJ_TRY(L.dev.alloc((size_t)2 * (t + 1) * sizeof(int32_t), st));
    PROJ_CUDA_TRY(cudaMemcpyAsync(L.dev.as<int32_t>(), L.seq_off.data(), (t + 1) * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, st));
    PROJ_CUDA_TRY(cudaMemcpyAsync(L.dev.as<int32_t>() + t + 1, L.lmer_off.data(),
                                  (t + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    return PROJ_OK;
}

// ---- Section 5 parameter choice (host) --------------------------------------

static double log_binom(int n, int r) {
    return lgamma(n + 1.0) - lgamma(r + 1.0) - lgamma(n - r + 1.0);
}

// Smallest m with 1 - B(s)^m >= q, B(s) = P[Bin(t_hat, p_hat) < s].
static int64_t trials_for(int l, int d, int k, int s, int t_hat, double q) {
    if (k < 1 || k > l - d || s < 1 || t_hat < 1 || !(q > 0.0 && q < 1.0)) return -1;
    const double lp = log_binom(l - d, k) - log_binom(l, k);
    const double p = exp(lp);
    double below = 0.0;
    for (int c = 0; c < s && c <= t_hat; ++c)
        below += exp(log_binom(t_hat, c) + c * lp + (t_hat - c) * log1p(-p));
    if (below >= 1.0) return -1;
    if (below <= 0.0) return 1;
    return (int64_t)ceil(log(1.0 - q) / log(below));
}

}  // namespace proj

using namespace proj;

extern "C" {

const char *projection_last_error(void) { return g_err; }

int64_t projection_packed_words(int64_t total_bases) {
    return total_bases <= 0 ? 0 : (total_bases + 15) / 16;
}

int projection_default_params(int t, const int64_t *lens, int l, int d, int *k, int *s, int *m) {
    clear_error();
    PROJ_REQUIRE(t >= 1 && lens && k && s && m, "bad arguments");
    PROJ_REQUIRE(l >= 1 && l <= 32 && d >= 0 && d < l, "need 0 <= d < l <= 32");
    int64_t x = 0;
    for (int i = 0; i < t; ++i) x += lens[i] >= l ? lens[i] - l + 1 : 0;
    if (*k == 0) *k = l - d - 1;
    PROJ_REQUIRE(*k >= 1 && *k <= l, "derived k = %d is out of range", *k);
    if (*s == 0) *s = (int)std::max<double>(3.0, ceil(2.0 * (double)x / pow(4.0, *k)));
    if (*m == 0) {
        const int64_t mm = trials_for(l, d, *k, *s, t, 0.95);
        PROJ_REQUIRE(mm >= 1 && mm <= (int64_t)1 << 24,
                     "no finite trial count for l=%d d=%d k=%d s=%d (k must be <= l-d)", l, d, *k,
                     *s);
        *m = (int)mm;
    }
    return PROJ_OK;
}

int projection_pack(const uint8_t *ascii_dev, int64_t total_bases, uint32_t *packed_dev,
                    int64_t *bad_index_dev, void *stream) {
    clear_error();
    PROJ_REQUIRE(total_bases >= 0, "total_bases must be >= 0");
    PROJ_REQUIRE(bad_index_dev && (total_bases == 0 || (ascii_dev && packed_dev)), "NULL buffer");
    return launch_pack(ascii_dev, total_bases, packed_dev, bad_index_dev, (cudaStream_t)stream);
}

int projection_background(const uint32_t *packed_dev, int64_t total_bases, double *bg_dev,
                          void *stream) {
    clear_error();
    PROJ_REQUIRE(total_bases >= 0 && bg_dev && (total_bases == 0 || packed_dev), "bad arguments");
    return launch_background(packed_dev, total_bases, bg_dev, (cudaStream_t)stream);
}

int projection_positions(uint64_t seed, int64_t trial_begin, int64_t n_trials, int l, int k,
                         uint8_t *pos_dev, void *stream) {
    clear_error();
    PROJ_REQUIRE(l >= 1 && l <= 32 && k >= 1 && k <= l, "need 1 <= k <= l <= 32");
    PROJ_REQUIRE(trial_begin >= 0 && n_trials >= 0, "trial range must be non-negative");
    PROJ_REQUIRE(n_trials == 0 || pos_dev, "pos_dev must not be NULL");
    return launch_positions(seed, trial_begin, n_trials, l, k, pos_dev, (cudaStream_t)stream);
}

int trial_hash(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l, int k, int s,
               uint64_t seed, int64_t trial_begin, int64_t n_trials, const int32_t *positions_in,
               uint8_t *positions_out_dev, uint32_t *counts_out_dev, int64_t cap_cand,
               int64_t cap_members, int32_t *cand_trial_dev, uint32_t *cand_key_dev,
               int32_t *cand_cnt_dev, int64_t *cand_off_dev, int32_t *members_dev,
               int64_t *totals_dev, void *stream) {
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    PROJ_REQUIRE(packed_dev != nullptr, "packed_dev must not be NULL");
    Layout L;
    PROJ_TRY(make_layout(seq_off, t, l, st, L));
    HashOut o;
    o.positions = positions_out_dev;
    o.counts = counts_out_dev;
    o.cap_cand = cap_cand;
    o.cap_members = cap_members;
    o.cand_trial = cand_trial_dev;
    o.cand_key = cand_key_dev;
    o.cand_cnt = cand_cnt_dev;
    o.cand_off = cand_off_dev;
    o.members = members_dev;
    o.totals = totals_dev;
    return run_trial_hash(packed_dev, L, k, s, seed, trial_begin, n_trials, positions_in, o, st);
}

int theta0_build(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l,
                 const int64_t *cand_off_dev, const int32_t *members_dev, int64_t C,
                 float pseudocount, float *theta0_dev, void *stream) {
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    PROJ_REQUIRE(C >= 0 && pseudocount >= 0.f, "need C >= 0 and pseudocount >= 0");
    PROJ_REQUIRE(C == 0 || (packed_dev && cand_off_dev && members_dev && theta0_dev), "NULL buffer");
    Layout L;
    PROJ_TRY(make_layout(seq_off, t, l, st, L));
    return launch_theta0(packed_dev, L, cand_off_dev, members_dev, C, pseudocount, theta0_dev, st);
}

int em_refine(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l,
              const double *bg_dev, const float *theta0_dev, int64_t C, int em_iters,
              float pseudocount, int precision, float *theta_out_dev, double *loglik_dev,
              int32_t *sites_out_dev, void *stream) {
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    PROJ_REQUIRE(C >= 0, "need C >= 0");
    PROJ_REQUIRE(C == 0 || (packed_dev && bg_dev && theta0_dev && theta_out_dev && loglik_dev),
                 "NULL buffer");
    Layout L;
    PROJ_TRY(make_layout(seq_off, t, l, st, L));
    PROJ_TRY(run_em(packed_dev, L, bg_dev, theta0_dev, C, em_iters, pseudocount, precision,
                    theta_out_dev, loglik_dev, st));
    if (sites_out_dev)
        PROJ_TRY(launch_cand_sites(packed_dev, L, bg_dev, theta_out_dev, C, sites_out_dev, st));
    return PROJ_OK;
}

int em_refine_zoops(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l,
                    const double *bg_dev, const float *theta0_dev, int64_t C, int em_iters,
                    float pseudocount, int precision, double site_prob, float *theta_out_dev,
                    double *loglik_dev, int32_t *sites_out_dev, void *stream) {
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    PROJ_REQUIRE(C >= 0, "need C >= 0");
    PROJ_REQUIRE(site_prob > 0.0 && site_prob <= 1.0, "need 0 < site_prob <= 1");
    PROJ_REQUIRE(C == 0 || (packed_dev && bg_dev && theta0_dev && theta_out_dev && loglik_dev),
                 "NULL buffer");
    Layout L;
    PROJ_TRY(make_layout(seq_off, t, l, st, L));
    PROJ_TRY(run_em(packed_dev, L, bg_dev, theta0_dev, C, em_iters, pseudocount, precision,
                    theta_out_dev, loglik_dev, st, site_prob));
    if (sites_out_dev)
        PROJ_TRY(launch_cand_sites(packed_dev, L, bg_dev, theta_out_dev, C, sites_out_dev, st));
    return PROJ_OK;
}

int projection_finalize(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l,
                        const double *bg_dev, const float *theta_dev, const double *loglik_dev,
                        int64_t C, int64_t *best_dev, int32_t *sites_dev, uint8_t *consensus_dev,
                        int32_t *score_dev, void *stream) {
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    PROJ_REQUIRE(C >= 0 && best_dev && sites_dev && consensus_dev && score_dev && packed_dev,
                 "bad arguments");
    PROJ_REQUIRE(C == 0 || (theta_dev && loglik_dev && bg_dev), "NULL buffer");
    Layout L;
    PROJ_TRY(make_layout(seq_off, t, l, st, L));
    return launch_finalize(packed_dev, L, bg_dev, theta_dev, loglik_dev, C, best_dev, sites_dev,
                           consensus_dev, score_dev, st);
}

// The winner's model, log-likelihood and (trial, key) gathered on the device so
// that the search's results come back in one copy.  sel (may be NULL) maps a
// refined candidate to its index in the full list.
__global__ void winner_kernel(const int64_t *__restrict__ best, const int64_t *__restrict__ sel,
                              const float *__restrict__ theta, int L4,
                              const double *__restrict__ ll, const int32_t *__restrict__ cand_trial,
                              const uint32_t *__restrict__ cand_key, int64_t *__restrict__ win,
                              double *__restrict__ ll_w, int32_t *__restrict__ trial_w,
                              uint32_t *__restrict__ key_w, float *__restrict__ pwm_w) {
    const int64_t b = *best;
    const int tid = threadIdx.x;
    if (b < 0) {
        if (tid == 0) {
            *win = -1;
            *ll_w = -INFINITY;
            *trial_w = -1;
            *key_w = 0u;
        }
        for (int q = tid; q < L4; q += blockDim.x) pwm_w[q] = 0.f;
        return;
    }
    const int64_t bo = sel ? sel[b] : b;
    if (tid == 0) {
        *win = bo;
        *ll_w = ll[b];
        *trial_w = cand_trial[bo];
        *key_w = cand_key[bo];
    }
    for (int q = tid; q < L4; q += blockDim.x) pwm_w[q] = theta[b * L4 + q];
}

// Fixed head of a search's small device buffer (read back in one copy); the
// sites [t], the winner's model [4l] and the consensus [l] follow it.
struct SearchHead {
    double bg[4];
    int64_t totals[2];
    int64_t best, win;
    double ll;
    int32_t score, err, trial;
    uint32_t key;
};

// Steps a2-a5 of a search plus the optional cap on refined buckets: counts
// every trial (sizing probe), builds the candidate list, and when `top` keeps
// fewer buckets than were enriched selects them (size descending, ties in
// (trial, key) order) and gathers their members into a compact list.
struct HashedSearch {
    HashState hstate;
    DevBuf off0, cand, compact;
    HashOut ho;
    int64_t C = 0, M = 0, R = 0;
    std::vector<int64_t> sel;      // kept candidate -> index in the full list (capped only)
    std::vector<int32_t> sel_cnt;
    const int64_t *r_off = nullptr;     // CSR of the refined buckets
    const int32_t *r_members = nullptr;
    int64_t *sel_dev = nullptr;         // device copy of sel (capped + table-only only)
};

static int hash_and_select(const uint32_t *packed, const Layout &L, int k, int s, uint64_t seed,
                           int m, int64_t top, int64_t *totals, const int64_t *bad_dev,
                           const uint8_t *ascii, HashedSearch &H, cudaStream_t st) {
    // pass sizes: count first, then size the candidate list exactly
    HashOut probe;
    PROJ_TRY(H.off0.alloc(sizeof(int64_t), st));
    probe.state = &H.hstate;  // the counting pass's partition and offsets, reused by the fill
    probe.totals = totals;
    probe.cand_off = H.off0.as<int64_t>();
    probe.count_only = true;
    probe.want_emit = top > 0;  // a capped search may build its table from the count
    PROJ_TRY(run_trial_hash(packed, L, k, s, seed, 0, m, nullptr, probe, st));
    int64_t tot_h[2], bad_h = -1;
    PROJ_CUDA_TRY(cudaMemcpyAsync(tot_h, totals, sizeof tot_h, cudaMemcpyDeviceToHost, st));
    if (bad_dev)
        PROJ_CUDA_TRY(cudaMemcpyAsync(&bad_h, bad_dev, sizeof bad_h, cudaMemcpyDeviceToHost, st));
    PROJ_CUDA_TRY(cudaStreamSynchronize(st));
    if (bad_h >= 0) {
        set_error("character %d at index %lld is not A/C/G/T", ascii ? (int)ascii[bad_h] : -1,
                  (long long)bad_h);
        return PROJ_EBADCHAR;
    }
    const int64_t C = tot_h[0], M = tot_h[1];
    H.C = C;
    H.M = M;

    // a capped search (top < C) needs the members of its kept buckets only: the
    // candidate table comes from the counting pass's lists and the kept
    // buckets' members are gathered afterwards
    const bool capped = top > 0 && C > top;
    const bool table_only = capped && H.hstate.emitted;
    const size_t cand_bytes = (size_t)C * (4 + 4 + 4) + (size_t)(C + 1) * 8 +
                              (table_only ? 0 : (size_t)M * 4) + 64;
    PROJ_TRY(H.cand.alloc(cand_bytes, st));
    HashOut &ho = H.ho;
    ho.cap_cand = C;
    ho.cap_members = table_only ? 0 : M;
    ho.cand_off = H.cand.as<int64_t>();
    ho.cand_trial = reinterpret_cast<int32_t *>(ho.cand_off + C + 1);
    ho.cand_key = reinterpret_cast<uint32_t *>(ho.cand_trial + C);
    ho.cand_cnt = reinterpret_cast<int32_t *>(ho.cand_key + C);
    ho.members = table_only ? nullptr : ho.cand_cnt + C;
    ho.totals = totals;
    ho.state = &H.hstate;
    ho.table_only = table_only;
    PROJ_TRY(run_trial_hash(packed, L, k, s, seed, 0, m, nullptr, ho, st));

    H.r_off = ho.cand_off;
    H.r_members = ho.members;
    H.R = C;
    if (capped) {
        PROJ_TRY(select_top(ho.cand_cnt, C, top, H.sel, H.sel_cnt, st));
        const int64_t n = (int64_t)H.sel.size();
        if (table_only) {
            // [new_off (n+1) | sel (n) | members]
            std::vector<int64_t> no_h(n + 1, 0);
            for (int64_t i = 0; i < n; ++i) no_h[i + 1] = no_h[i] + H.sel_cnt[i];
            PROJ_TRY(H.compact.alloc((size_t)(2 * n + 1) * 8 + (size_t)no_h[n] * 4 + 64, st));
            int64_t *no = H.compact.as<int64_t>();
            int64_t *sd = no + n + 1;
            int32_t *nm = reinterpret_cast<int32_t *>(sd + n);
            PROJ_CUDA_TRY(cudaMemcpyAsync(no, no_h.data(), (n + 1) * 8, cudaMemcpyHostToDevice, st));
            PROJ_CUDA_TRY(cudaMemcpyAsync(sd, H.sel.data(), n * 8, cudaMemcpyHostToDevice, st));
            PROJ_TRY(run_kept_table(H.hstate, sd, n, ho.cand_trial, ho.cand_key, st));
            PROJ_TRY(run_gather_members(packed, L, H.hstate, k, seed, sd, n, ho.cand_trial,
                                        ho.cand_key, no, nm, st));
            H.r_off = no;
            H.r_members = nm;
            H.sel_dev = sd;
        } else {
            int64_t *no = nullptr;
            int32_t *nm = nullptr;
            PROJ_TRY(gather_selected(H.sel, H.sel_cnt, ho.cand_off, ho.members, H.compact, &no, &nm,
                                     st));
            H.r_off = no;
            H.r_members = nm;
        }
        H.R = n;
    }
    return PROJ_OK;
}

static int find_impl(const uint32_t *packed, const int64_t *seq_off, int t, int l, int d, int k,
                     int s, int m, uint64_t seed, int em_iters, float pseudocount, int precision,
                     int64_t top, projection_result *out, cudaStream_t st, double gamma = 1.0,
                     const int64_t *bad_dev = nullptr, const uint8_t *ascii = nullptr) {
    // bad_dev: the pack kernel's first non-ACGT index (or -1), checked at the
    // first synchronisation of the search
    PROJ_REQUIRE(packed != nullptr, "packed input must not be NULL");
    PROJ_REQUIRE(d >= 0 && d < l, "need 0 <= d < l");
    Layout L;
    PROJ_TRY(make_layout(seq_off, t, l, st, L));
    {
        std::vector<int64_t> lens(t);
        for (int i = 0; i < t; ++i) lens[i] = seq_off[i + 1] - seq_off[i];
        PROJ_TRY(projection_default_params(t, lens.data(), l, d, &k, &s, &m));
    }
    PROJ_REQUIRE(k >= 1 && k <= l && k <= 10, "need 1 <= k <= min(l, 10), got %d", k);
    PROJ_REQUIRE(s >= 1 && m >= 1, "need s >= 1 and m >= 1");
    out->t = t; out->l = l; out->k = k; out->s = s; out->m = m;

    DevBuf small;  // SearchHead | sites[t] | pwm[4l] | consensus[l]
    const size_t small_bytes = sizeof(SearchHead) + (size_t)t * 4 + (size_t)16 * l + (size_t)l;
    PROJ_TRY(small.alloc(small_bytes + 16, st));
    PROJ_CUDA_TRY(cudaMemsetAsync(small.as<void>(), 0, sizeof(SearchHead), st));
    SearchHead *head = small.as<SearchHead>();
    double *bg = head->bg;
    int64_t *totals = head->totals;
    int64_t *best = &head->best;
    int32_t *score = &head->score;
    int32_t *sites = reinterpret_cast<int32_t *>(head + 1);
    float *pwm_w = reinterpret_cast<float *>(sites + t);
    uint8_t *cons = reinterpret_cast<uint8_t *>(pwm_w + 4 * l);
    PROJ_TRY(launch_background(packed, L.total, bg, st));

    HashedSearch hsr;
    PROJ_TRY(hash_and_select(packed, L, k, s, seed, m, top, totals, bad_dev, ascii, hsr, st));
    const int64_t C = hsr.C, R = hsr.R;
    out->n_candidates = C;
    out->n_members = hsr.M;
    const int64_t *r_off = hsr.r_off;
    const int32_t *r_members = hsr.r_members;
    const std::vector<int64_t> &sel = hsr.sel;
    HashOut &ho = hsr.ho;
    out->n_refined = R;

    DevBuf model;
    PROJ_TRY(model.alloc((size_t)R * 4 * l * sizeof(float) + (size_t)R * sizeof(double) + 16, st));
    double *ll = model.as<double>();
    float *theta = reinterpret_cast<float *>(ll + R);
    PROJ_TRY(launch_theta0(packed, L, r_off, r_members, R, pseudocount, theta, st));
    PROJ_TRY(run_em(packed, L, bg, theta, R, em_iters, pseudocount, precision, theta, ll, st, gamma,
                    &head->err));
    PROJ_TRY(launch_finalize(packed, L, bg, theta, ll, R, best, sites, cons, score, st));
    DevBuf sel_dev;  // refined candidate -> index in the full list (top selection only)
    if (!sel.empty()) {
        PROJ_TRY(sel_dev.alloc(sel.size() * sizeof(int64_t), st));
        PROJ_CUDA_TRY(cudaMemcpyAsync(sel_dev.as<int64_t>(), sel.data(), sel.size() * sizeof(int64_t),
                                      cudaMemcpyHostToDevice, st));
    }
    winner_kernel<<<1, 128, 0, st>>>(best, sel.empty() ? nullptr : sel_dev.as<int64_t>(), theta,
                                     4 * l, ll, ho.cand_trial, ho.cand_key, &head->win, &head->ll,
                                     &head->trial, &head->key, pwm_w);
    PROJ_LAUNCH_CHECK("winner_kernel");

    std::vector<uint8_t> res(small_bytes);
    PROJ_CUDA_TRY(cudaMemcpyAsync(res.data(), small.as<void>(), small_bytes, cudaMemcpyDeviceToHost, st));
    PROJ_CUDA_TRY(cudaStreamSynchronize(st));
    SearchHead h;
    memcpy(&h, res.data(), sizeof h);
    if (h.err) {
        set_error("a bounded wait for tensor-core completion expired in em_tc_kernel");
        return PROJ_ETIMEOUT;
    }
    out->win_index = h.win;
    out->pwm = (float *)calloc((size_t)4 * l, sizeof(float));
    out->consensus = (char *)calloc((size_t)l + 1, 1);
    out->sites = (int32_t *)calloc((size_t)t, sizeof(int32_t));
    if (!out->pwm || !out->consensus || !out->sites) {
        set_error("host allocation failed");
        return PROJ_ENOMEM;
    }
    memcpy(out->sites, res.data() + sizeof(SearchHead), (size_t)t * 4);
    memcpy(out->pwm, res.data() + sizeof(SearchHead) + (size_t)t * 4, (size_t)16 * l);
    memcpy(out->consensus, res.data() + sizeof(SearchHead) + (size_t)t * 4 + (size_t)16 * l, (size_t)l);
    out->score = h.score;
    out->loglik = h.ll;
    out->win_trial = h.trial;
    out->win_key = h.key;
    out->consensus[l] = 0;
    if (h.win < 0) {
        out->loglik = -INFINITY;
        out->win_trial = -1;
        out->win_key = 0;
    }
    return PROJ_OK;
}


// Kept buckets' (trial, key, size) in selection order.
__global__ void sel_table_kernel(const int64_t *__restrict__ sel, int64_t n,
                                 const int32_t *__restrict__ cand_trial,
                                 const uint32_t *__restrict__ cand_key,
                                 const int32_t *__restrict__ cand_cnt, int64_t *__restrict__ o_idx,
                                 int32_t *__restrict__ o_trial, uint32_t *__restrict__ o_key,
                                 int32_t *__restrict__ o_cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t c = sel[i];
    o_idx[i] = c;
    o_trial[i] = cand_trial[c];
    o_key[i] = cand_key[c];
    o_cnt[i] = cand_cnt[c];
}

int trial_hash_top(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l, int k, int s,
                   uint64_t seed, int64_t n_trials, int64_t top, int64_t cap_members,
                   int64_t *sel_index_dev, int32_t *cand_trial_dev, uint32_t *cand_key_dev,
                   int32_t *cand_cnt_dev, int64_t *cand_off_dev, int32_t *members_dev,
                   int64_t *totals_dev, void *stream) {
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    PROJ_REQUIRE(packed_dev != nullptr && totals_dev != nullptr, "NULL buffer");
    PROJ_REQUIRE(top >= 1, "need top >= 1");
    PROJ_REQUIRE(n_trials >= 1 && n_trials <= (1 << 24), "need 1 <= n_trials <= 2^24");
    PROJ_REQUIRE(sel_index_dev && cand_trial_dev && cand_key_dev && cand_cnt_dev && cand_off_dev,
                 "NULL candidate buffer");
    PROJ_REQUIRE(cap_members >= 0 && (cap_members == 0 || members_dev), "bad member buffer");
    Layout L;
    PROJ_TRY(make_layout(seq_off, t, l, st, L));
    DevBuf tb;
    PROJ_TRY(tb.alloc(2 * sizeof(int64_t), st));
    HashedSearch H;
    PROJ_TRY(hash_and_select(packed_dev, L, k, s, seed, (int)n_trials, top, tb.as<int64_t>(),
                             nullptr, nullptr, H, st));
    if (H.sel.empty() && H.C > 0) {
        // every enriched bucket is kept: put them in the same size order
        PROJ_TRY(select_top(H.ho.cand_cnt, H.C, H.C, H.sel, H.sel_cnt, st));
        int64_t *no = nullptr;
        int32_t *nm = nullptr;
        PROJ_TRY(gather_selected(H.sel, H.sel_cnt, H.ho.cand_off, H.ho.members, H.compact, &no,
                                 &nm, st));
        H.r_off = no;
        H.r_members = nm;
    }
    const int64_t R = (int64_t)H.sel.size();
    int64_t kept = 0;
    for (int32_t c : H.sel_cnt) kept += c;
    const int64_t tot[4] = {H.C, H.M, R, kept};
    PROJ_CUDA_TRY(cudaMemcpyAsync(totals_dev, tot, sizeof tot, cudaMemcpyHostToDevice, st));
    if (kept > cap_members) {
        PROJ_CUDA_TRY(cudaStreamSynchronize(st));
        set_error("the kept buckets hold %lld members, above cap_members = %lld", (long long)kept,
                  (long long)cap_members);
        return PROJ_ECAPACITY;
    }
    if (R > 0) {
        DevBuf sd;
        PROJ_TRY(sd.alloc((size_t)R * 8, st));
        PROJ_CUDA_TRY(cudaMemcpyAsync(sd.as<int64_t>(), H.sel.data(), R * 8, cudaMemcpyHostToDevice,
                                      st));
        sel_table_kernel<<<(unsigned)((R + 255) / 256), 256, 0, st>>>(
            sd.as<int64_t>(), R, H.ho.cand_trial, H.ho.cand_key, H.ho.cand_cnt, sel_index_dev,
            cand_trial_dev, cand_key_dev, cand_cnt_dev);
        PROJ_LAUNCH_CHECK("sel_table_kernel");
        PROJ_CUDA_TRY(cudaMemcpyAsync(cand_off_dev, H.r_off, (R + 1) * 8, cudaMemcpyDeviceToDevice,
                                      st));
        if (kept > 0)
            PROJ_CUDA_TRY(cudaMemcpyAsync(members_dev, H.r_members, kept * 4,
                                          cudaMemcpyDeviceToDevice, st));
    } else {
        PROJ_CUDA_TRY(cudaMemsetAsync(cand_off_dev, 0, sizeof(int64_t), st));
    }
    PROJ_CUDA_TRY(cudaStreamSynchronize(st));
    return PROJ_OK;
}

static void result_init(projection_result *out) {
    memset(out, 0, sizeof *out);
    out->win_index = -1;
    out->win_trial = -1;
}

int projection_find_packed(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l,
                           int d, int k, int s, int m, uint64_t seed, int em_iters,
                           float pseudocount, int precision, projection_result *out,
                           void *stream) {
    clear_error();
    if (!out) { set_error("out must not be NULL"); return PROJ_EINVAL; }
    result_init(out);
    const int rc = find_impl(packed_dev, seq_off, t, l, d, k, s, m, seed, em_iters, pseudocount,
                             precision, 0, out, (cudaStream_t)stream);
    out->status = rc;
    return rc;
}

int projection_find_packed_top(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l,
                               int d, int k, int s, int m, uint64_t seed, int em_iters,
                               float pseudocount, int precision, int64_t top,
                               projection_result *out, void *stream) {
    clear_error();
    if (!out) { set_error("out must not be NULL"); return PROJ_EINVAL; }
    result_init(out);
    if (top < 0) { set_error("top must be >= 0"); out->status = PROJ_EINVAL; return PROJ_EINVAL; }
    const int rc = find_impl(packed_dev, seq_off, t, l, d, k, s, m, seed, em_iters, pseudocount,
                             precision, top, out, (cudaStream_t)stream);
    out->status = rc;
    return rc;
}

int projection_find_packed_zoops(const uint32_t *packed_dev, const int64_t *seq_off, int t,
                                 int l, int d, int k, int s, int m, uint64_t seed, int em_iters,
                                 float pseudocount, int precision, double site_prob, int64_t top,
                                 projection_result *out, void *stream) {
    clear_error();
    if (!out) { set_error("out must not be NULL"); return PROJ_EINVAL; }
    result_init(out);
    if (top < 0 || !(site_prob > 0.0 && site_prob <= 1.0)) {
        set_error("need top >= 0 and 0 < site_prob <= 1");
        out->status = PROJ_EINVAL;
        return PROJ_EINVAL;
    }
    const int rc = find_impl(packed_dev, seq_off, t, l, d, k, s, m, seed, em_iters, pseudocount,
                             precision, top, out, (cudaStream_t)stream, site_prob);
    out->status = rc;
    return rc;
}


static int find_host(const uint8_t *ascii, const int64_t *seq_off, int t, int l, int d, int k,
                     int s, int m, uint64_t seed, int em_iters, float pseudocount, int precision,
                     int64_t top, projection_result *out, void *stream) {
    clear_error();
    if (!out) { set_error("out must not be NULL"); return PROJ_EINVAL; }
    result_init(out);
    cudaStream_t st = (cudaStream_t)stream;
    auto fail = [&](int rc) { out->status = rc; return rc; };
    if (!ascii || !seq_off || t < 1) { set_error("bad input arrays"); return fail(PROJ_EINVAL); }
    const int64_t total = seq_off[t];
    if (total < 0 || total >= ((int64_t)1 << 31)) { set_error("bad total length"); return fail(PROJ_EINVAL); }
    DevBuf in;
    int rc = in.alloc((size_t)total + (size_t)projection_packed_words(total) * 4 + 64, st);
    if (rc) return fail(rc);
    uint8_t *ascii_dev = in.as<uint8_t>();
    int64_t *bad = reinterpret_cast<int64_t *>(ascii_dev + ((total + 15) & ~(int64_t)15));
    uint32_t *packed = reinterpret_cast<uint32_t *>(bad + 2);
    cudaError_t e = cudaMemcpyAsync(ascii_dev, ascii, (size_t)total, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { set_error("H2D copy failed: %s", cudaGetErrorString(e)); return fail(PROJ_ECUDA); }
    rc = launch_pack(ascii_dev, total, packed, bad, st);
    if (rc) return fail(rc);
    rc = find_impl(packed, seq_off, t, l, d, k, s, m, seed, em_iters, pseudocount, precision, top,
                   out, st, 1.0, bad, ascii);
    out->status = rc;
    return rc;
}

int projection_find(const uint8_t *ascii, const int64_t *seq_off, int t, int l, int d, int k,
                    int s, int m, uint64_t seed, int em_iters, float pseudocount, int precision,
                    projection_result *out, void *stream) {
    return find_host(ascii, seq_off, t, l, d, k, s, m, seed, em_iters, pseudocount, precision, 0,
                     out, stream);
}

int projection_find_top(const uint8_t *ascii, const int64_t *seq_off, int t, int l, int d, int k,
                        int s, int m, uint64_t seed, int em_iters, float pseudocount,
                        int precision, int64_t top, projection_result *out, void *stream) {
    if (top < 0) {
        set_error("top must be >= 0");
        if (out) { result_init(out); out->status = PROJ_EINVAL; }
        return PROJ_EINVAL;
    }
    return find_host(ascii, seq_off, t, l, d, k, s, m, seed, em_iters, pseudocount, precision, top,
                     out, stream);
}

int projection_find_batch(const uint8_t *ascii, const int64_t *seq_off, const int *inst_seq,
                          int n_inst, const int *l, const int *d, const int *k, const int *s,
                          const int *m, const uint64_t *seed, int em_iters, float pseudocount,
                          int precision, projection_result *out, void *stream) {
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    if (!out || n_inst < 1) { set_error("need out[] and n_inst >= 1"); return PROJ_EINVAL; }
    for (int i = 0; i < n_inst; ++i) result_init(&out[i]);
    auto fail = [&](int rc) {
        for (int i = 0; i < n_inst; ++i) out[i].status = rc;
        return rc;
    };
    if (!ascii || !seq_off || !inst_seq || !l || !d || !k || !s || !m || !seed) {
        set_error("NULL argument");
        return fail(PROJ_EINVAL);
    }
    if (precision != PROJ_EM_BF16_SPLIT) {
        set_error("batched searches run the tensor-core EM (PROJ_EM_BF16_SPLIT); use "
                  "projection_find per instance for PROJ_EM_FP32");
        return fail(PROJ_ENOTSUP);
    }
    if (!(pseudocount > 0.f) || em_iters < 0 || em_iters > 1000) {
        set_error("need pseudocount > 0 and 0 <= em_iters <= 1000");
        return fail(PROJ_EINVAL);
    }
    const int n_seq = inst_seq[n_inst];
    if (inst_seq[0] != 0 || n_seq < 1 || seq_off[0] != 0) { set_error("bad inst_seq/seq_off"); return fail(PROJ_EINVAL); }
    const int64_t total = seq_off[n_seq];
    if (total >= ((int64_t)1 << 31)) { set_error("input longer than 2^31 - 1 bases"); return fail(PROJ_EINVAL); }

    // ---- host-side plan: per-instance parameters and offsets
    std::vector<int> K(n_inst), S(n_inst), Mt(n_inst);
    std::vector<int32_t> offs;           // per instance: [rel (t+1) | lmer (t+1) | global (t+1)]
    std::vector<int64_t> off_pos(n_inst), base_range(2 * n_inst);
    std::vector<int64_t> word_lo(n_inst), nwords_i(n_inst), xs(n_inst);
    int l_max = 1, t_sum = 0, l_sum = 0;
    for (int i = 0; i < n_inst; ++i) {
        const int sb = inst_seq[i], se = inst_seq[i + 1], t = se - sb;
        if (t < 1 || l[i] < 1 || l[i] > 32 || d[i] < 0 || d[i] >= l[i]) {
            set_error("instance %d: need t >= 1, 1 <= l <= 32, 0 <= d < l", i);
            return fail(PROJ_EINVAL);
        }
        std::vector<int64_t> lens(t);
        for (int j = 0; j < t; ++j) {
            lens[j] = seq_off[sb + j + 1] - seq_off[sb + j];
            if (lens[j] < l[i]) {
                set_error("instance %d: sequence %d is shorter than l = %d", i, j, l[i]);
                return fail(PROJ_EINVAL);
            }
        }
        K[i] = k[i]; S[i] = s[i]; Mt[i] = m[i];
        int rc = projection_default_params(t, lens.data(), l[i], d[i], &K[i], &S[i], &Mt[i]);
        if (rc) return fail(rc);
        if (K[i] < 1 || K[i] > 10 || K[i] > l[i]) {
            set_error("instance %d: need 1 <= k <= min(l, 10), got %d", i, K[i]);
            return fail(PROJ_EINVAL);
        }
        word_lo[i] = seq_off[sb] >> 4;
        nwords_i[i] = ((seq_off[se] + 15) >> 4) - word_lo[i];
        base_range[2 * i] = seq_off[sb];
        base_range[2 * i + 1] = seq_off[se];
        off_pos[i] = (int64_t)offs.size();
        int64_t x = 0;
        for (int j = 0; j <= t; ++j) offs.push_back((int32_t)(seq_off[sb + j] - 16 * word_lo[i]));
        offs.push_back(0);
        for (int j = 0; j < t; ++j) { x += lens[j] - l[i] + 1; offs.push_back((int32_t)x); }
        for (int j = 0; j <= t; ++j) offs.push_back((int32_t)seq_off[sb + j]);
        xs[i] = x;
        l_max = std::max(l_max, l[i]);
        t_sum += t;
        l_sum += l[i];
        out[i].t = t; out[i].l = l[i]; out[i].k = K[i]; out[i].s = S[i]; out[i].m = Mt[i];
    }
    const int stride = 4 * l_max;

    // ---- device: input, offsets, background
    DevBuf in, offb, ranges, bgb;
    int rc = in.alloc((size_t)total + (size_t)projection_packed_words(total) * 4 + 64, st);
    if (rc) return fail(rc);
    uint8_t *ascii_dev = in.as<uint8_t>();
    int64_t *bad = reinterpret_cast<int64_t *>(ascii_dev + ((total + 15) & ~(int64_t)15));
    uint32_t *packed = reinterpret_cast<uint32_t *>(bad + 2);
    const int64_t nwords = (total + 15) / 16;
#define BATCH_TRY(expr) do { int rc_ = (expr); if (rc_) return fail(rc_); } while (0)
#define BATCH_CUDA(expr) do { cudaError_t e_ = (expr); if (e_ != cudaSuccess) { set_error("%s: %s", #expr, cudaGetErrorString(e_)); return fail(PROJ_ECUDA); } } while (0)
    BATCH_CUDA(cudaMemcpyAsync(ascii_dev, ascii, (size_t)total, cudaMemcpyHostToDevice, st));
    BATCH_TRY(launch_pack(ascii_dev, total, packed, bad, st));
    BATCH_TRY(offb.alloc(offs.size() * sizeof(int32_t), st));
    BATCH_CUDA(cudaMemcpyAsync(offb.as<int32_t>(), offs.data(), offs.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, st));
    BATCH_TRY(ranges.alloc(base_range.size() * sizeof(int64_t), st));
    BATCH_CUDA(cudaMemcpyAsync(ranges.as<int64_t>(), base_range.data(),
                               base_range.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    BATCH_TRY(bgb.alloc((size_t)n_inst * 4 * sizeof(double), st));
    BATCH_TRY(launch_background_batch(packed, ranges.as<int64_t>(), n_inst, bgb.as<double>(), st));
    {
        int64_t bad_h = -1;
        BATCH_CUDA(cudaMemcpyAsync(&bad_h, bad, 8, cudaMemcpyDeviceToHost, st));
        BATCH_CUDA(cudaStreamSynchronize(st));
        if (bad_h >= 0) {
            set_error("character %d at index %lld is not A/C/G/T", (int)ascii[bad_h], (long long)bad_h);
            return fail(PROJ_EBADCHAR);
        }
    }

    // ---- all trials of all instances
    std::vector<HashInstSpec> spec(n_inst);
    for (int i = 0; i < n_inst; ++i) {
        const int t = inst_seq[i + 1] - inst_seq[i];
        HashInstSpec &q = spec[i];
        q.packed = packed + word_lo[i];
        q.nwords = nwords_i[i];
        q.seq_off_rel = offb.as<int32_t>() + off_pos[i];
        q.lmer_off = q.seq_off_rel + (t + 1);
        q.t = t; q.l = l[i]; q.k = K[i]; q.s = S[i]; q.m = Mt[i];
        q.x = (int)xs[i];
        q.seed = seed[i];
    }
    HashBatchOut H;
    BATCH_TRY(run_hash_batch(spec, H, st));
    const int64_t C = H.C;

    // ---- theta^0, EM, finalise for all candidates
    std::vector<BatchInst> bi(n_inst);
    std::vector<EmInstHost> eh(n_inst);
    std::vector<EmInst> ei(n_inst);
    int64_t sites_off = 0, cons_off = 0;
    for (int i = 0; i < n_inst; ++i) {
        const int t = inst_seq[i + 1] - inst_seq[i];
        const int32_t *rel = offb.as<int32_t>() + off_pos[i];
        bi[i].seq_off = rel + 2 * (t + 1);  // global positions
        bi[i].lmer_off = rel + (t + 1);
        bi[i].bg = bgb.as<double>() + 4 * i;
        bi[i].t = t;
        bi[i].l = l[i];
        bi[i].cand_begin = H.cand_begin[i];
        bi[i].C = H.n_cand[i];
        bi[i].sites_off = sites_off;
        bi[i].cons_off = cons_off;
        sites_off += t;
        cons_off += l[i];
        eh[i].t = t; eh[i].l = l[i]; eh[i].C = H.n_cand[i]; eh[i].cand_begin = H.cand_begin[i];
        eh[i].lmers = xs[i];
        eh[i].seq_off = offs.data() + off_pos[i] + 2 * (t + 1);  // global positions
        ei[i].seq_off = bi[i].seq_off; ei[i].bg = bi[i].bg; ei[i].t = t; ei[i].l = l[i];
        ei[i].cand_begin = H.cand_begin[i];
        ei[i].gamma = 1.0;  // OOPS
        out[i].n_candidates = H.n_cand[i];
        out[i].n_members = H.n_mem[i];
    }
    DevBuf bib, eib, model, res;
    BATCH_TRY(bib.alloc(bi.size() * sizeof(BatchInst), st));
    BATCH_TRY(eib.alloc(ei.size() * sizeof(EmInst), st));
    BATCH_CUDA(cudaMemcpyAsync(bib.as<BatchInst>(), bi.data(), bi.size() * sizeof(BatchInst),
                               cudaMemcpyHostToDevice, st));
    BATCH_CUDA(cudaMemcpyAsync(eib.as<EmInst>(), ei.data(), ei.size() * sizeof(EmInst),
                               cudaMemcpyHostToDevice, st));
    BATCH_TRY(model.alloc((size_t)C * stride * sizeof(float) + (size_t)C * sizeof(double) + 64, st));
    double *ll = model.as<double>();
    float *theta = reinterpret_cast<float *>(ll + C);
    BATCH_TRY(launch_theta0_batch(packed, nwords, bib.as<BatchInst>(), n_inst, H.cand_off(),
                                  H.members(), C, pseudocount, stride, theta, st));
    const size_t res_bytes = (size_t)n_inst * (8 + 4) + (size_t)t_sum * 4 + (size_t)l_sum + 64;
    BATCH_TRY(res.alloc(res_bytes, st));
    int64_t *best = res.as<int64_t>();
    int32_t *score = reinterpret_cast<int32_t *>(best + n_inst);
    int32_t *sites = score + n_inst;
    uint8_t *cons = reinterpret_cast<uint8_t *>(sites + t_sum);
    // EM iterations and the per-instance finalisation replay as one graph
    EmTcRun run;
    BATCH_TRY(em_tc_prepare(packed, nwords, eh, eib.as<EmInst>(), theta, C, stride, run, st));
    BATCH_TRY(run_as_graph(kGraphBatchTail, st, [&](cudaStream_t cs) {
        PROJ_TRY(em_tc_enqueue(run, em_iters, pseudocount, theta, ll, cs));
        return launch_finalize_batch(packed, nwords, bib.as<BatchInst>(), n_inst, theta, stride, ll,
                                     best, sites, cons, score, cs);
    }));
    BATCH_TRY(em_tc_finish(run, st));
    std::vector<unsigned char> hres(res_bytes);
    BATCH_CUDA(cudaMemcpyAsync(hres.data(), res.as<unsigned char>(), res_bytes,
                               cudaMemcpyDeviceToHost, st));
    BATCH_CUDA(cudaStreamSynchronize(st));
    const int64_t *hbest = reinterpret_cast<const int64_t *>(hres.data());
    const int32_t *hscore = reinterpret_cast<const int32_t *>(hbest + n_inst);
    const int32_t *hsites = hscore + n_inst;
    const uint8_t *hcons = reinterpret_cast<const uint8_t *>(hsites + t_sum);
    // the winners' models, log-likelihoods, trials and keys
    std::vector<int64_t> widx;
    for (int i = 0; i < n_inst; ++i)
        if (hbest[i] >= 0) widx.push_back(H.cand_begin[i] + hbest[i]);
    std::vector<float> wpwm(widx.size() * stride);
    std::vector<double> wll(widx.size());
    std::vector<int32_t> wtrial(widx.size());
    std::vector<uint32_t> wkey(widx.size());
    for (size_t q = 0; q < widx.size(); ++q) {
        BATCH_CUDA(cudaMemcpyAsync(&wpwm[q * stride], theta + widx[q] * stride, stride * sizeof(float),
                                   cudaMemcpyDeviceToHost, st));
        BATCH_CUDA(cudaMemcpyAsync(&wll[q], ll + widx[q], 8, cudaMemcpyDeviceToHost, st));
        BATCH_CUDA(cudaMemcpyAsync(&wtrial[q], H.cand_trial() + widx[q], 4, cudaMemcpyDeviceToHost, st));
        BATCH_CUDA(cudaMemcpyAsync(&wkey[q], H.cand_key() + widx[q], 4, cudaMemcpyDeviceToHost, st));
    }
    BATCH_CUDA(cudaStreamSynchronize(st));
    size_t q = 0;
    int64_t so = 0, co = 0;
    for (int i = 0; i < n_inst; ++i) {
        projection_result &r = out[i];
        const int t = r.t, li = r.l;
        r.pwm = (float *)calloc((size_t)4 * li, sizeof(float));
        r.consensus = (char *)calloc((size_t)li + 1, 1);
        r.sites = (int32_t *)calloc((size_t)t, sizeof(int32_t));
        if (!r.pwm || !r.consensus || !r.sites) { set_error("host allocation failed"); return fail(PROJ_ENOMEM); }
        memcpy(r.sites, hsites + so, (size_t)t * 4);
        memcpy(r.consensus, hcons + co, (size_t)li);
        r.consensus[li] = 0;
        r.score = hscore[i];
        r.win_index = hbest[i];
        if (hbest[i] >= 0) {
            memcpy(r.pwm, &wpwm[q * stride], (size_t)4 * li * sizeof(float));
            r.loglik = wll[q];
            r.win_trial = wtrial[q];
            r.win_key = wkey[q];
            ++q;
        } else {
            r.loglik = -INFINITY;
        }
        r.status = PROJ_OK;
        so += t;
        co += li;
    }
#undef BATCH_TRY
#undef BATCH_CUDA
    return PROJ_OK;
}

void projection_result_free(projection_result *r) {
    if (!r) return;
    free(r->pwm);
    free(r->consensus);
    free(r->sites);
    r->pwm = nullptr;
    r->consensus = nullptr;
    r->sites = nullptr;
}

}  // extern "C"
