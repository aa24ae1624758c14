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
              void *stream) {
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    PROJ_REQUIRE(C >= 0, "need C >= 0");
    PROJ_REQUIRE(C == 0 || (packed_dev && bg_dev && theta0_dev && theta_out_dev && loglik_dev),
                 "NULL buffer");
    Layout L;
    PROJ_TRY(make_layout(seq_off, t, l, st, L));
    return run_em(packed_dev, L, bg_dev, theta0_dev, C, em_iters, pseudocount, precision,
                  theta_out_dev, loglik_dev, st);
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

static int find_impl(const uint32_t *packed, const int64_t *seq_off, int t, int l, int d, int k,
                     int s, int m, uint64_t seed, int em_iters, float pseudocount, int precision,
                     projection_result *out, cudaStream_t st) {
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

    DevBuf small;  // bg[4] | totals[2] | best | score | sites[t] | consensus[l]
    const size_t small_bytes = 4 * 8 + 2 * 8 + 8 + 8 + (size_t)t * 4 + (size_t)l + 16;
    PROJ_TRY(small.alloc(small_bytes, st));
    double *bg = small.as<double>();
    int64_t *totals = reinterpret_cast<int64_t *>(bg + 4);
    int64_t *best = totals + 2;
    int32_t *score = reinterpret_cast<int32_t *>(best + 1);
    int32_t *sites = score + 2;
    uint8_t *cons = reinterpret_cast<uint8_t *>(sites + t);
    PROJ_TRY(launch_background(packed, L.total, bg, st));

    // pass sizes: count first, then size the candidate list exactly
    HashOut probe;
    DevBuf off0;
    PROJ_TRY(off0.alloc(sizeof(int64_t), st));
    probe.totals = totals;
    probe.cand_off = off0.as<int64_t>();
    probe.count_only = true;
    PROJ_TRY(run_trial_hash(packed, L, k, s, seed, 0, m, nullptr, probe, st));
    int64_t tot_h[2];
    PROJ_CUDA_TRY(cudaMemcpyAsync(tot_h, totals, sizeof tot_h, cudaMemcpyDeviceToHost, st));
    PROJ_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t C = tot_h[0], M = tot_h[1];
    out->n_candidates = C;
    out->n_members = M;

    DevBuf cand;
    const size_t cand_bytes = (size_t)C * (4 + 4 + 4) + (size_t)(C + 1) * 8 + (size_t)M * 4 + 64;
    PROJ_TRY(cand.alloc(cand_bytes, st));
    HashOut ho;
    ho.cap_cand = C;
    ho.cap_members = M;
    ho.cand_off = cand.as<int64_t>();
    ho.cand_trial = reinterpret_cast<int32_t *>(ho.cand_off + C + 1);
    ho.cand_key = reinterpret_cast<uint32_t *>(ho.cand_trial + C);
    ho.cand_cnt = reinterpret_cast<int32_t *>(ho.cand_key + C);
    ho.members = ho.cand_cnt + C;
    ho.totals = totals;
    PROJ_TRY(run_trial_hash(packed, L, k, s, seed, 0, m, nullptr, ho, st));

    DevBuf model;
    PROJ_TRY(model.alloc((size_t)C * 4 * l * sizeof(float) + (size_t)C * sizeof(double) + 16, st));
    double *ll = model.as<double>();
    float *theta = reinterpret_cast<float *>(ll + C);
    PROJ_TRY(launch_theta0(packed, L, ho.cand_off, ho.members, C, pseudocount, theta, st));
    PROJ_TRY(run_em(packed, L, bg, theta, C, em_iters, pseudocount, precision, theta, ll, st));
    PROJ_TRY(launch_finalize(packed, L, bg, theta, ll, C, best, sites, cons, score, st));

    int64_t b = -1;
    PROJ_CUDA_TRY(cudaMemcpyAsync(&b, best, sizeof b, cudaMemcpyDeviceToHost, st));
    PROJ_CUDA_TRY(cudaStreamSynchronize(st));
    out->win_index = b;
    out->pwm = (float *)calloc((size_t)4 * l, sizeof(float));
    out->consensus = (char *)calloc((size_t)l + 1, 1);
    out->sites = (int32_t *)calloc((size_t)t, sizeof(int32_t));
    if (!out->pwm || !out->consensus || !out->sites) {
        set_error("host allocation failed");
        return PROJ_ENOMEM;
    }
    PROJ_CUDA_TRY(cudaMemcpyAsync(out->sites, sites, (size_t)t * 4, cudaMemcpyDeviceToHost, st));
    PROJ_CUDA_TRY(cudaMemcpyAsync(out->consensus, cons, (size_t)l, cudaMemcpyDeviceToHost, st));
    PROJ_CUDA_TRY(cudaMemcpyAsync(&out->score, score, 4, cudaMemcpyDeviceToHost, st));
    if (b >= 0) {
        PROJ_CUDA_TRY(cudaMemcpyAsync(out->pwm, theta + b * 4 * l, (size_t)4 * l * sizeof(float),
                                      cudaMemcpyDeviceToHost, st));
        PROJ_CUDA_TRY(cudaMemcpyAsync(&out->loglik, ll + b, 8, cudaMemcpyDeviceToHost, st));
        PROJ_CUDA_TRY(cudaMemcpyAsync(&out->win_trial, ho.cand_trial + b, 4, cudaMemcpyDeviceToHost, st));
        PROJ_CUDA_TRY(cudaMemcpyAsync(&out->win_key, ho.cand_key + b, 4, cudaMemcpyDeviceToHost, st));
    }
    PROJ_CUDA_TRY(cudaStreamSynchronize(st));
    out->consensus[l] = 0;
    if (b < 0) {
        out->loglik = -INFINITY;
        out->win_trial = -1;
        out->win_key = 0;
    }
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
                             precision, out, (cudaStream_t)stream);
    out->status = rc;
    return rc;
}

int projection_find(const uint8_t *ascii, const int64_t *seq_off, int t, int l, int d, int k,
                    int s, int m, uint64_t seed, int em_iters, float pseudocount, int precision,
                    projection_result *out, void *stream) {
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
    int64_t bad_h = -1;
    e = cudaMemcpyAsync(&bad_h, bad, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { set_error("D2H copy failed: %s", cudaGetErrorString(e)); return fail(PROJ_ECUDA); }
    if (bad_h >= 0) {
        set_error("character %d at index %lld is not A/C/G/T", (int)ascii[bad_h], (long long)bad_h);
        return fail(PROJ_EBADCHAR);
    }
    rc = find_impl(packed, seq_off, t, l, d, k, s, m, seed, em_iters, pseudocount, precision, out, st);
    out->status = rc;
    return rc;
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
