// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the C ABI (that is include/projection.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <vector>

#include "../../include/projection.h"

namespace proj {

// ---------------------------------------------------------------------------
// Error reporting (thread-local message, status codes of projection.h)
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);
void clear_error();

#define PROJ_CUDA_TRY(expr)                                                              \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            ::proj::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),    \
                              __FILE__, __LINE__);                                       \
            return e_ == cudaErrorMemoryAllocation ? PROJ_ENOMEM : PROJ_ECUDA;           \
        }                                                                                \
    } while (0)

#define PROJ_LAUNCH_CHECK(what)                                                          \
    do {                                                                                 \
        cudaError_t e_ = cudaGetLastError();                                             \
        if (e_ != cudaSuccess) {                                                         \
            ::proj::set_error("launch of %s failed: %s", what, cudaGetErrorString(e_));   \
            return PROJ_ECUDA;                                                           \
        }                                                                                \
    } while (0)

#define PROJ_TRY(expr)                                                                   \
    do {                                                                                 \
        int st_ = (expr);                                                                \
        if (st_ != PROJ_OK) return st_;                                                  \
    } while (0)

#define PROJ_REQUIRE(cond, ...)                                                          \
    do {                                                                                 \
        if (!(cond)) {                                                                   \
            ::proj::set_error(__VA_ARGS__);                                              \
            return PROJ_EINVAL;                                                          \
        }                                                                                \
    } while (0)

// Stream-ordered device scratch: cudaMallocAsync on construction, cudaFreeAsync
// on destruction (same stream).
class DevBuf {
  public:
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    int alloc(size_t bytes, cudaStream_t st);
    void release();
    template <class T> T *as() const { return reinterpret_cast<T *>(ptr_); }
    size_t bytes() const { return bytes_; }

  private:
    void *ptr_ = nullptr;
    size_t bytes_ = 0;
    cudaStream_t st_ = nullptr;
};

// Validated sequence layout of one input (host side), with int32 device copies
// of the base offsets and l-mer offsets.
struct Layout {
    int t = 0, l = 0;
    int64_t total = 0;        // concatenated bases
    int64_t x = 0;            // l-mers
    int max_ns = 0;           // most l-mers in one sequence
    int64_t nwords = 0;       // packed 32-bit words
    std::vector<int32_t> seq_off, lmer_off;  // t+1 each
    DevBuf dev;               // [seq_off | lmer_off] as int32
    const int32_t *seq_off_dev() const { return dev.as<int32_t>(); }
    const int32_t *lmer_off_dev() const { return dev.as<int32_t>() + (t + 1); }
};

// Checks t, l and the offsets; fills `L` and uploads the offsets on `st`.
int make_layout(const int64_t *seq_off, int t, int l, cudaStream_t st, Layout &L);

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files; all asynchronous on `st`)
// ---------------------------------------------------------------------------
int launch_pack(const uint8_t *ascii, int64_t total, uint32_t *packed, int64_t *bad,
                cudaStream_t st);
int launch_background(const uint32_t *packed, int64_t total, double *bg, cudaStream_t st);
int launch_positions(uint64_t seed, int64_t trial_begin, int64_t n_trials, int l, int k,
                     uint8_t *pos, cudaStream_t st);

// What a counting call of run_trial_hash computed, kept for the filling call of
// the same search (same input, k, s, seed and trials) so that the key-range
// partition, the per-unit counts and their offsets are not computed twice.
struct HashState {
    DevBuf meta, part_buf;
    DevBuf emit_buf;     // the counting pass's per-unit enriched (key, size) lists
    DevBuf pos_buf;      // every trial's projected positions [n_trials][k]
    bool valid = false;
    bool emitted = false;  // emit_buf holds the lists (counting call had want_emit)
    // what the member gather of selected buckets needs from the counting call
    int parts = 1, hb = 0, n_chunks = 0;
    int nt = 0;                      // threads per bucket-kernel CTA chosen by the counting call
    bool partitioned = false;
    const uint16_t *prel = nullptr;    // partitioned mode: keys grouped by part per chunk
    const uint16_t *plid = nullptr;    //                   chunk-local l-mer ids
    const int32_t *pstart = nullptr;   //                   part starts per (trial, chunk)
    const uint8_t *pos_tab = nullptr;  // positions of the call's trials (null: drawn in-kernel)
    // a table-only filling call: each unit's first candidate index, and the units
    int64_t n_units = 0, trial_begin = 0;
    const int64_t *cand_base = nullptr;
};

struct HashOut {
    HashState *state = nullptr;     // optional: filled by a count_only call, reused after
    uint8_t *positions = nullptr;   // [n_trials][k] or null
    uint32_t *counts = nullptr;     // [n_trials][4^k] or null
    int64_t cap_cand = 0, cap_members = 0;
    int32_t *cand_trial = nullptr;
    uint32_t *cand_key = nullptr;
    int32_t *cand_cnt = nullptr;
    int64_t *cand_off = nullptr;
    int32_t *members = nullptr;
    int64_t *totals = nullptr;      // device int64[2]
    bool count_only = false;        // stop after the totals (sizing probe)
    bool want_emit = false;         // counting call: also keep each unit's enriched lists
    bool table_only = false;        // filling call: only the candidates' sizes, from those
                                    // lists, and no members (the caller fills in the
                                    // trials and keys of the ones it keeps and gathers
                                    // their members)
};

// Both passes of the bucket kernels plus the scan between them.
int run_trial_hash(const uint32_t *packed, const Layout &L, int k, int s, uint64_t seed,
                   int64_t trial_begin, int64_t n_trials, const int32_t *positions_in,
                   const HashOut &out, cudaStream_t st);

// Members (ascending l-mer ids) of n selected candidates of a search whose
// counting call kept its state: candidate sel[i] = (cand_trial, cand_key) of
// the full list; its members go to new_members[new_off[i] .. new_off[i+1]).
// Trials and keys of the kept candidates sel[0..n) (indices into the list of
// all enriched buckets) after a table-only filling call, written at those indices.
int run_kept_table(const HashState &hs, const int64_t *sel, int64_t n, int32_t *cand_trial,
                   uint32_t *cand_key, cudaStream_t st);
int run_gather_members(const uint32_t *packed, const Layout &L, const HashState &hs, int k,
                       uint64_t seed, const int64_t *sel, int64_t n, const int32_t *cand_trial,
                       const uint32_t *cand_key, const int64_t *new_off, int32_t *new_members,
                       cudaStream_t st);

// ---- batched motif searches ------------------------------------------------
// One instance of a batched hash: its packed words start at `packed`
// (positions in seq_off_rel are relative to that word), device offsets.
struct HashInstSpec {
    const uint32_t *packed = nullptr;
    int64_t nwords = 0;
    const int32_t *seq_off_rel = nullptr;  // device [t+1]
    const int32_t *lmer_off = nullptr;     // device [t+1]
    int t = 0, l = 0, k = 0, s = 0, x = 0, m = 0;
    uint64_t seed = 0;
};

// Candidate lists of all instances of a batch, in (instance, trial, key) order.
struct HashBatchOut {
    std::vector<int64_t> cand_begin, n_cand, mem_begin, n_mem;  // per instance
    int64_t C = 0, M = 0;
    DevBuf cand;  // [cand_off (C+1) | cand_trial | cand_key | cand_cnt | members]
    int64_t *cand_off() const { return cand.as<int64_t>(); }
    int32_t *cand_trial() const { return reinterpret_cast<int32_t *>(cand_off() + C + 1); }
    uint32_t *cand_key() const { return reinterpret_cast<uint32_t *>(cand_trial() + C); }
    int32_t *cand_cnt() const { return reinterpret_cast<int32_t *>(cand_key() + C); }
    int32_t *members() const { return cand_cnt() + C; }
};

// All trials of all instances: one count launch, a scan, one synchronisation
// to size the lists, one fill launch.
int run_hash_batch(const std::vector<HashInstSpec> &spec, HashBatchOut &out, cudaStream_t st);

// Per-instance view used by the batched theta^0, background and finalise
// kernels (device copy); positions are into the whole packed input.
struct BatchInst {
    const int32_t *seq_off;   // [t+1]
    const int32_t *lmer_off;  // [t+1]
    const double *bg;         // [4]
    int t, l;
    int64_t cand_begin, C;
    int64_t sites_off;        // first entry of its sites in the batch's sites array
    int64_t cons_off;         // first letter of its consensus in the batch's consensus array
};
int launch_theta0_batch(const uint32_t *packed, int64_t nwords, const BatchInst *inst, int n_inst,
                        const int64_t *cand_off, const int32_t *members, int64_t C, float beta,
                        int stride, float *theta0, cudaStream_t st);
int launch_finalize_batch(const uint32_t *packed, int64_t nwords, const BatchInst *inst,
                          int n_inst, const float *theta, int stride, const double *ll,
                          int64_t *best, int32_t *sites, uint8_t *consensus, int32_t *score,
                          cudaStream_t st);
int launch_background_batch(const uint32_t *packed, const int64_t *base_range, int n_inst,
                            double *bg, cudaStream_t st);

// All-pairs enrichment (csrc/allpairs.cu) for DNA (alphabet 4, packed input)
// or proteins (alphabet 20, byte codes).
int run_allpairs(const uint32_t *packed, const uint8_t *codes, int alphabet, const Layout &L,
                 int k, int s, uint64_t seed, int64_t trial_begin, int64_t n_trials,
                 int64_t cap_cand, int64_t cap_members, int32_t *cand_trial_dev,
                 uint32_t *cand_key_dev, int32_t *cand_cnt_dev, int64_t *cand_off_dev,
                 int32_t *members_dev, int64_t *totals_dev, cudaStream_t st);

int launch_theta0(const uint32_t *packed, const Layout &L, const int64_t *cand_off,
                  const int32_t *members, int64_t C, float beta, float *theta0, cudaStream_t st);

// err_dev: when not NULL, the tensor-core path's timeout flag (int, nonzero =
// PROJ_ETIMEOUT) is copied there on the stream and not checked here, so the
// caller can read it with its results instead of synchronising in between.
int run_em(const uint32_t *packed, const Layout &L, const double *bg, const float *theta0,
           int64_t C, int iters, float beta, int precision, float *theta_out, double *ll,
           cudaStream_t st, double gamma = 1.0, int *err_dev = nullptr);

// Per candidate c < C and sequence i: sites[c][i] = the first start j that
// maximises r(i,j) under theta[c], scored in FP64 (Definition 1's start vector).
int launch_cand_sites(const uint32_t *packed, const Layout &L, const double *bg,
                      const float *theta, int64_t C, int32_t *sites, cudaStream_t st);
int launch_finalize(const uint32_t *packed, const Layout &L, const double *bg,
                    const float *theta, const double *ll, int64_t C, int64_t *best,
                    int32_t *sites, uint8_t *consensus, int32_t *score, cudaStream_t st);

int sm_count();

// The `top` largest candidates (size desc, index asc) and their sizes; empty
// when top <= 0.  Synchronises `st`.
int select_top(const int32_t *cnt_dev, int64_t C, int64_t top, std::vector<int64_t> &sel,
               std::vector<int32_t> &sel_cnt, cudaStream_t st);
// Compact CSR list (offsets, members) of the selected candidates in out_buf.
int gather_selected(const std::vector<int64_t> &sel, const std::vector<int32_t> &sel_cnt,
                    const int64_t *cand_off, const int32_t *members, DevBuf &out_buf,
                    int64_t **new_off, int32_t **new_members, cudaStream_t st);

// Event pair around one kernel launch while tracing is enabled
// (projection_trace_enable); a no-op otherwise.
class TraceSpan {
  public:
    TraceSpan(const char *name, cudaStream_t st);
    ~TraceSpan() { end(); }
    void end();

  private:
    int slot_ = -1;
    cudaStream_t st_;
};
bool trace_active();

// Runs `body` (launches only: no allocation, no synchronisation) as a CUDA
// graph on `st`: captured on a private stream, its executable graph kept per
// (host thread, device, slot) and updated in place on the next call.
// PROJ_GRAPHS=0 in the environment runs `body` directly on `st` instead.
int run_as_graph(int slot, cudaStream_t st, const std::function<int(cudaStream_t)> &body);
enum GraphSlot { kGraphEm = 0, kGraphBatchTail = 1 };

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64-bit products with multipliers 0xD2511F53 / 0xCD9E8D57, the high
// halves xored with the other counter words and the round key, the key
// advanced by the Weyl increments 0x9E3779B9 / 0xBB67AE85 after each round.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a0 = c[0], a2 = c[2];
        const uint32_t hi0 = __umulhi(0xD2511F53u, a0), lo0 = 0xD2511F53u * a0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, a2), lo1 = 0xCD9E8D57u * a2;
        c[0] = hi1 ^ c[1] ^ k0;
        c[1] = lo1;
        c[2] = hi0 ^ c[3] ^ k1;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Algorithm 2 step 2a: l-k distinct excluded positions by a partial
// Fisher-Yates shuffle of 0..l-1; word w of the Philox stream with counter
// (trial lo, w/4, trial hi, 0) picks the swap partner i + floor(u*(l-i)/2^32).
// Writes the k kept positions in increasing order.
__device__ inline void draw_positions(uint64_t seed, uint64_t trial, int l, int k, int *pos) {
    uint8_t perm[32];
    for (int i = 0; i < l; ++i) perm[i] = (uint8_t)i;
    uint32_t c[4] = {0u, 0u, 0u, 0u};
    for (int i = 0; i < l - k; ++i) {
        if ((i & 3) == 0) {
            c[0] = (uint32_t)trial;
            c[1] = (uint32_t)(i >> 2);
            c[2] = (uint32_t)(trial >> 32);
            c[3] = 0u;
            philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        }
        const uint32_t u = c[i & 3];
        const int j = i + (int)(((uint64_t)u * (uint64_t)(l - i)) >> 32);
        const uint8_t tmp = perm[i];
        perm[i] = perm[j];
        perm[j] = tmp;
    }
    uint32_t excl = 0u;
    for (int i = 0; i < l - k; ++i) excl |= 1u << perm[i];
    int q = 0;
    for (int p = 0; p < l; ++p)
        if (!((excl >> p) & 1u)) pos[q++] = p;
}

// 2-bit code of base b (A0 C1 T2 G3) from packed words, 0 beyond the input.
__device__ __forceinline__ uint32_t code_at(const uint32_t *__restrict__ w, int64_t nwords,
                                            int64_t b) {
    const int64_t wi = b >> 4;
    return wi < nwords ? (__ldg(w + wi) >> (2 * (b & 15))) & 3u : 0u;
}

// 64-bit window holding the codes of bases b0 .. b0+31 (bits 2p..2p+1 = base
// b0+p) from a word array `w` whose valid words are [0, nwords); words past the
// end read as zero.
__device__ __forceinline__ uint64_t window64(const uint32_t *w, int64_t nwords, int64_t b0) {
    const int64_t wi = b0 >> 4;
    const int sh = (int)(b0 & 15) * 2;
    const uint64_t w0 = wi < nwords ? w[wi] : 0u;
    const uint64_t w1 = wi + 1 < nwords ? w[wi + 1] : 0u;
    const uint64_t w2 = wi + 2 < nwords ? w[wi + 2] : 0u;
    const uint64_t lo = w0 | (w1 << 32);
    return sh ? ((lo >> sh) | (w2 << (64 - sh))) : lo;
}

}  // namespace proj
