/*
 * projection.h -- C ABI of the GB300 (sm_103a) PROJECTION motif finder.
 *
 * The method is PROJECTION (Buhler & Tompa) as restated by Clemente, Cabarle &
 * Adorna, "PROJECTION Algorithm for Motif Finding on GPUs" (arXiv 1605.06904):
 * for each of m random trials, project every l-mer of the t input sequences
 * onto k of its l positions (Section 5, random projection h_k), hash the
 * projected k-mer in base 4 (Section 6, A:0 C:1 T:2 G:3, most significant
 * digit first) into 4^k buckets (Algorithm 2 step 2c), keep the buckets holding
 * at least s l-mers (Algorithm 2 step 3; Section 6), and refine each enriched
 * bucket's position weight matrix by EM (Section 5.1) under the
 * one-occurrence-per-sequence model.
 *
 * Conventions for every call:
 *   - Pointers named *_dev are device pointers on the current CUDA device;
 *     every other pointer is host memory.  The caller owns all buffers passed
 *     in; the library never frees them.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Device work
 *     is enqueued on it; calls return once their work is enqueued unless the
 *     description says they synchronise.
 *   - Scratch memory is allocated stream-ordered on `stream` from a memory
 *     pool the library creates per device (freed blocks stay cached in that
 *     pool for reuse) and freed on the same stream before the call returns.
 *   - Return value: PROJ_OK (0) or a negative PROJ_E* status.  No C++
 *     exception crosses this boundary.  projection_last_error() returns a
 *     human-readable message for the calling thread's last failure.
 *   - Sequences are given in linear form (Section 6): one concatenated buffer
 *     plus seq_off[t+1], sequence i occupying [seq_off[i], seq_off[i+1]).
 *     Every sequence must hold at least one l-mer (n_i >= l).  The concatenated
 *     length and the number of l-mers x = sum_i (n_i - l + 1) are below 2^31.
 *   - Global l-mer id: l-mer S_{i,j} (0-based start j in sequence i) has id
 *     sum_{i'<i} (n_{i'} - l + 1) + j.
 *   - PWMs are float [l][4] in code order A, C, T, G; columns sum to 1.
 *   - Limits: 1 <= k <= l <= 32, k <= 10, 1 <= t.
 */
#ifndef PROJECTION_H
#define PROJECTION_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PROJ_OK 0
#define PROJ_EINVAL (-1)    /* an argument is out of range */
#define PROJ_ENOMEM (-2)    /* a device allocation failed */
#define PROJ_ECAPACITY (-3) /* a caller buffer is too small (needed size written back) */
#define PROJ_ECUDA (-4)     /* a CUDA runtime call failed */
#define PROJ_ETIMEOUT (-5)  /* a bounded device wait expired */
#define PROJ_EBADCHAR (-6)  /* the input holds a character other than A/C/G/T */
#define PROJ_ENOTSUP (-7)   /* parameters outside what the kernels implement */

/* ---- EM arithmetic ------------------------------------------------------ */
#define PROJ_EM_FP32 0       /* scores, exp and M-step sums in FP32 on CUDA cores */
#define PROJ_EM_BF16_SPLIT 1 /* scoring and M-step contractions on tcgen05 tensor cores,
                                BF16 hi+lo split operands, FP32 accumulation */

/* Message of the calling thread's most recent failure ("" if none). */
const char *projection_last_error(void);

/* ---- host-side helpers (no device work) -------------------------------- */

/* Number of 32-bit words projection_pack writes for `total_bases` bases:
 * ceil(total_bases / 16).  Base b sits in word b/16 at bits 2*(b%16)..+1. */
int64_t projection_packed_words(int64_t total_bases);

/* Algorithm 2 step 1 ("if not specified") with the Section 5 choices: an
 * input of 0 in *k, *s or *m is replaced by k = l-d-1,
 * s = max(3, ceil(2 x / 4^k)) (twice the mean bucket size, floored at the
 * paper's empirical 3), m = ceil(log(1-q) / log B(s)) with q = 0.95,
 * t_hat = t, p_hat = C(l-d,k)/C(l,k), B(s) = P[Binomial(t_hat, p_hat) < s].
 * lens[t] are the sequence lengths.  Returns PROJ_EINVAL if no valid value
 * exists (e.g. k > l-d makes p_hat = 0) or the bound exceeds 2^24 trials. */
int projection_default_params(int t, const int64_t *lens, int l, int d, int *k, int *s, int *m);

/* ---- step a1: pack (Section 6, linear 2-bit form) ----------------------- */

/* Packs `total_bases` ASCII bases (A/C/G/T, either case) into 2-bit codes
 * A0 C1 T2 G3, ceil(total_bases/16) words, high bits of the last word zero.
 * *bad_index_dev (int64, device) receives -1, or the smallest index of a
 * character that is not A/C/G/T (its word is then unspecified). */
int projection_pack(const uint8_t *ascii_dev, int64_t total_bases, uint32_t *packed_dev,
                    int64_t *bad_index_dev, void *stream);

/* Background model of Section 5.1 (column 0 of theta): the 0-order base
 * frequencies of the whole packed input, as double[4] in code order; a base
 * that never occurs is counted once.  Writes bg_dev[0..3]. */
int projection_background(const uint32_t *packed_dev, int64_t total_bases, double *bg_dev,
                          void *stream);

/* ---- step a2: projection positions (Algorithm 2 step 2a) ---------------- */

/* For trials trial_begin .. trial_begin+n_trials-1 writes the k projected
 * positions (0-based, increasing) to pos_dev[n][k] (uint8).  The l-k excluded
 * positions are distinct, chosen by a partial Fisher-Yates shuffle of 0..l-1
 * driven by Philox4x32-10 with key (seed lo, seed hi) and counter
 * (trial lo, block, trial hi, 0); word w of the draw picks swap partner
 * i + floor(u_w * (l - i) / 2^32). */
int projection_positions(uint64_t seed, int64_t trial_begin, int64_t n_trials, int l, int k,
                         uint8_t *pos_dev, void *stream);

/* ---- steps a2-a5: project, hash, count, enrich (Algorithm 2 steps 2-3) -- */

/* Runs trials trial_begin .. trial_begin+n_trials-1 in one pass.
 *   packed_dev     2-bit input from projection_pack
 *   seq_off        host int64[t+1] base offsets of the sequences
 *   positions_in   host int32[k]: if not NULL every trial uses these projected
 *                  positions instead of drawing them (worked examples, tests)
 *   positions_out_dev  device uint8[n_trials][k] or NULL
 *   counts_out_dev device uint32[n_trials][4^k] bucket sizes, or NULL
 * Output: the enriched buckets (size >= s) of all trials in (trial, key)
 * order, as a CSR list in caller buffers of capacity cap_cand / cap_members:
 *   cand_trial_dev int32[cap_cand], cand_key_dev uint32[cap_cand],
 *   cand_cnt_dev int32[cap_cand], cand_off_dev int64[cap_cand+1]
 *   (members of candidate c are members_dev[cand_off[c] .. cand_off[c+1]),
 *   members_dev int32[cap_members] global l-mer ids, ascending per candidate.
 * totals_dev (int64[2], device) receives the full candidate and member counts
 * even when they exceed the capacities; entries beyond a capacity are not
 * written and the caller must retry with larger buffers.  Asynchronous. */
int trial_hash(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l, int k, int s,
               uint64_t seed, int64_t trial_begin, int64_t n_trials, const int32_t *positions_in,
               uint8_t *positions_out_dev, uint32_t *counts_out_dev, int64_t cap_cand,
               int64_t cap_members, int32_t *cand_trial_dev, uint32_t *cand_key_dev,
               int32_t *cand_cnt_dev, int64_t *cand_off_dev, int32_t *members_dev,
               int64_t *totals_dev, void *stream);

/* Algorithm 2 steps 2-3 for trials 0 .. n_trials-1, keeping only the `top`
 * largest enriched buckets: the paper enriches buckets by the threshold s
 * alone (Algorithm 2 step 3); inputs with 10^6..10^7 enriched buckets refine
 * a bounded number of them.  Buckets are ordered by size, largest first, ties
 * in (trial, key) order, and R = min(top, C) are kept, C = all enriched.
 * Outputs, in that order (device buffers of top entries, cand_off top+1):
 *   sel_index_dev  int64: the bucket's index in trial_hash's (trial, key) list
 *   cand_trial_dev, cand_key_dev, cand_cnt_dev: as trial_hash
 *   cand_off_dev   int64[R+1] offsets of the kept buckets' members in
 *   members_dev    int32[cap_members]: global l-mer ids, ascending per bucket.
 * totals_dev int64[4] receives C, the members of all enriched buckets, R and
 * the members of the kept ones; PROJ_ECAPACITY (nothing else written) when
 * the last exceeds cap_members.  top >= 1.  Synchronises `stream`. */
int trial_hash_top(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l, int k, int s,
                   uint64_t seed, int64_t n_trials, int64_t top, int64_t cap_members,
                   int64_t *sel_index_dev, int32_t *cand_trial_dev, uint32_t *cand_key_dev,
                   int32_t *cand_cnt_dev, int64_t *cand_off_dev, int32_t *members_dev,
                   int64_t *totals_dev, void *stream);

/* The paper has no counterpart to this call; it serves callers of this library
 * that cannot allocate device memory -- a service that gave all device memory
 * to its own pool allocator at start-up, or a latency-critical path that must
 * not pay for an allocation (cudaMalloc may synchronise the device).
 * Same arguments, outputs and status codes as trial_hash, but no device memory
 * is allocated: the scratch lives in one fixed array of
 * PROJ_NOALLOC_SCRATCH_BYTES inside the library, held by every GPU that loads
 * the library until the process exits.  Needs
 *   a(8 (t+1)) + a(8 n_units) + a(16 n_units) + a(8 cap_members)   bytes,
 * a(v) = v rounded up to a multiple of 256, n_units = n_trials * parts with
 *   parts = 1                 when 4^k <= 32768 (u32 counters in one CTA),
 *   parts = max(1, 4^k/65536) when 4^k > 32768 and x <= 65535 (u16 counters),
 *   parts = 4^k / 32768       otherwise (u32 counters, key-range parts),
 * x = number of l-mers.  A request above the limit returns PROJ_ECAPACITY with
 * a message and launches nothing.  All calls share the array: calls whose
 * device work overlaps (other streams, other threads) race and must be
 * serialised by the caller.  The first call on each device looks up the
 * array's device address (once, with that device current) and keeps it for
 * the life of the process (no cudaDeviceReset in between); make that first
 * call before any stream capture.  The sequence offsets reach the device
 * inside kernel parameters, so no device work reads seq_off after the call
 * returns. */
#define PROJ_NOALLOC_SCRATCH_BYTES (8u << 20)
int trial_hash_noalloc(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l, int k,
                       int s, uint64_t seed, int64_t trial_begin, int64_t n_trials,
                       const int32_t *positions_in, uint8_t *positions_out_dev,
                       uint32_t *counts_out_dev, int64_t cap_cand, int64_t cap_members,
                       int32_t *cand_trial_dev, uint32_t *cand_key_dev, int32_t *cand_cnt_dev,
                       int64_t *cand_off_dev, int32_t *members_dev, int64_t *totals_dev,
                       void *stream);

/* ---- step a6: initial model theta^0 (Example 1, Figure 4) -------------- */

/* theta0_dev[c][p][a] = (#members of candidate c with base a at position p
 * + pseudocount) / (cnt_c + 4 pseudocount), for c < C, from the CSR list of
 * trial_hash (cand_off_dev, members_dev). */
int theta0_build(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l,
                 const int64_t *cand_off_dev, const int32_t *members_dev, int64_t C,
                 float pseudocount, float *theta0_dev, void *stream);

/* ---- steps a7-a8: EM refinement (Section 5.1, OOPS) --------------------- */

/* For each of C starting models theta0_dev[C][l][4] runs em_iters EM
 * iterations and a final E-step.  With W_c[p][a] = log theta_c[p][a] -
 * log bg[a] and r(i,j) = sum_p W_c[p][x_{i,j+p}]:
 *   E-step: z(i,j) = exp(r(i,j)) / sum_j' exp(r(i,j'))   (per sequence)
 *   M-step: theta[p][a] = (sum_{i,j} z(i,j) [x_{i,j+p} = a] + pseudocount)
 *                         / (t + 4 pseudocount)
 * theta_out_dev[C][l][4] receives the model after em_iters M-steps (it may
 * alias theta0_dev) and loglik_dev[C] (double) the log-likelihood ratio of
 * that model against the background,
 *   LL = sum_i [ log sum_j exp r(i,j) - log(n_i - l + 1) ],
 * per-sequence log-sum-exp in FP32, sum over sequences in FP64.
 * bg_dev: double[4] from projection_background.  precision: PROJ_EM_FP32 or
 * PROJ_EM_BF16_SPLIT.  pseudocount must be > 0.
 * sites_out_dev: int32[C][t] or NULL.  When given, row c receives the start
 * vector of Definition 1 (Section 2) under candidate c's final model: per
 * sequence i the first 0-based start j maximising r(i,j), evaluated in FP64
 * from theta_out_dev (as projection_finalize does for the winner). */
int em_refine(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l,
              const double *bg_dev, const float *theta0_dev, int64_t C, int em_iters,
              float pseudocount, int precision, float *theta_out_dev, double *loglik_dev,
              int32_t *sites_out_dev, void *stream);

/* The same refinement under the zero-or-one-occurrence model (ZOOPS, the
 * second search model named in Section 2): a sequence holds one site with
 * probability site_prob (fixed, 0 < site_prob <= 1), uniform over its starts,
 * or none.  Per sequence i with ns_i starts the log-likelihood ratio is
 *     L_i = log[(1 - site_prob) + (site_prob / ns_i) sum_j e^{r(i,j)}],
 * the posterior of a site at j is (site_prob / ns_i) e^{r(i,j)} / e^{L_i}, and the
 * M-step is theta_p(a) = (sum z [x = a] + pseudocount) / (sum z + 4 pseudocount).
 * site_prob = 1 is the OOPS model of em_refine (up to rounding).  Arguments,
 * layouts and errors as em_refine (sites_out_dev: the first start of highest
 * score in every sequence, as there); EINVAL for site_prob outside (0, 1]. */
int em_refine_zoops(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l,
                    const double *bg_dev, const float *theta0_dev, int64_t C, int em_iters,
                    float pseudocount, int precision, double site_prob, float *theta_out_dev,
                    double *loglik_dev, int32_t *sites_out_dev, void *stream);

/* ---- step a9: rank and finalise ----------------------------------------- */

/* Picks the best candidate (largest loglik, FP64; a tie goes to the smaller
 * index, i.e. the earlier (trial, key)) and, for its model theta_dev[best]:
 *   sites_dev int32[t]   per sequence the first start maximising r(i,j),
 *                        evaluated in FP64;
 *   consensus_dev uint8[l] ASCII consensus, per column the base of largest
 *                        weight, ties to the lowest code (A, C, T, G);
 *   score_dev int32[1]   Score(s, DNA) of Section 2 for those sites;
 *   best_dev int64[1]    the chosen candidate index (-1 when C == 0). */
int projection_finalize(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l,
                        const double *bg_dev, const float *theta_dev, const double *loglik_dev,
                        int64_t C, int64_t *best_dev, int32_t *sites_dev, uint8_t *consensus_dev,
                        int32_t *score_dev, void *stream);

/* ---- whole path --------------------------------------------------------- */

typedef struct {
    int status;            /* PROJ_OK or the failing status */
    int t, l, k, s, m;     /* resolved parameters */
    int64_t n_candidates;  /* enriched buckets over all trials */
    int64_t n_members;     /* l-mers in them */
    int64_t win_index;     /* index of the winner in (trial, key) order, -1 if none */
    int win_trial;
    uint32_t win_key;
    double loglik;         /* winner's log-likelihood ratio */
    int score;             /* Score(s, DNA) of the winner's sites */
    float *pwm;            /* [l][4], allocated by the library */
    char *consensus;       /* l letters + NUL, allocated by the library */
    int32_t *sites;        /* [t] 0-based starts, allocated by the library */
    int64_t n_refined;     /* candidates refined by EM (n_candidates, or `top`) */
} projection_result;

/* The paper's problem statement (Algorithm 2: INPUT t sequences, l, n, d;
 * OUTPUT motif): from host ASCII sequences in linear form (ascii[seq_off[t]],
 * seq_off[t+1]) runs pack, k/s/m defaults (0 = derive), m trials of
 * projection + hashing, theta^0 and EM for every enriched bucket, and ranking.
 * Copies in, computes, copies the small result out, and synchronises
 * `stream`.  `out` is filled on success and on failure (out->status); its
 * arrays are released by projection_result_free. */
int projection_find(const uint8_t *ascii, const int64_t *seq_off, int t, int l, int d, int k,
                    int s, int m, uint64_t seed, int em_iters, float pseudocount, int precision,
                    projection_result *out, void *stream);

/* As projection_find, with the input already packed on the device. */
int projection_find_packed(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l,
                           int d, int k, int s, int m, uint64_t seed, int em_iters,
                           float pseudocount, int precision, projection_result *out,
                           void *stream);

/* As projection_find / projection_find_packed, refining only the `top`
 * enriched buckets with the most member l-mers (ties keep (trial, key) order;
 * top = 0 refines all).  The paper ranks buckets only by the threshold s; the
 * cap bounds EM work on serving-scale inputs with 10^6..10^7 enriched buckets.
 * out->n_candidates counts all enriched buckets, out->n_refined the refined
 * ones, out->win_index indexes the full (trial, key)-ordered list. */
int projection_find_top(const uint8_t *ascii, const int64_t *seq_off, int t, int l, int d, int k,
                        int s, int m, uint64_t seed, int em_iters, float pseudocount,
                        int precision, int64_t top, projection_result *out, void *stream);
int projection_find_packed_top(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l,
                               int d, int k, int s, int m, uint64_t seed, int em_iters,
                               float pseudocount, int precision, int64_t top,
                               projection_result *out, void *stream);

/* projection_find_packed_top with the EM of em_refine_zoops (site_prob in
 * (0, 1]; top = 0 refines every enriched bucket).  Sites are reported as in
 * the OOPS search: per sequence the first start of highest score under the
 * winning model (a caller that wants "no site" decisions thresholds the
 * posterior itself). */
int projection_find_packed_zoops(const uint32_t *packed_dev, const int64_t *seq_off, int t,
                                 int l, int d, int k, int s, int m, uint64_t seed, int em_iters,
                                 float pseudocount, int precision, double site_prob, int64_t top,
                                 projection_result *out, void *stream);

/* Batched serving: n_inst independent searches in one call.  Instance i owns
 * sequences inst_seq[i] .. inst_seq[i+1]-1 of the linear input (ascii,
 * seq_off[inst_seq[n_inst]+1]); its parameters are l[i], d[i], k[i], s[i], m[i]
 * (0 = the Section 5 choice) and seed[i].  The trials of all instances are
 * hashed in one launch, the candidates of all instances are refined by one
 * EM launch per iteration (work items of 128 candidates x a range of their own
 * instance's sequences, taken in turn by a persistent grid), and each
 * instance is ranked on its own.  Requires precision = PROJ_EM_BF16_SPLIT.
 * Synchronises `stream`.  out[n_inst] is filled like projection_find's; each
 * entry is released by projection_result_free. */
int projection_find_batch(const uint8_t *ascii, const int64_t *seq_off, const int *inst_seq,
                          int n_inst, const int *l, const int *d, const int *k, const int *s,
                          const int *m, const uint64_t *seed, int em_iters, float pseudocount,
                          int precision, projection_result *out, void *stream);

void projection_result_free(projection_result *r);

/* ---- low-memory enrichment by all-pairs comparison ---------------------- */

/* Algorithm 2 steps 2-3 without the 4^k bucket table: per trial every l-mer's
 * projected k-mer is compared with those of all x l-mers of the trial
 * (PROJECTION2 of Section 5.2; the pairwise compare of Section 6's
 * CUDA-PROJECTION), O(x) memory and O(x^2) work per trial.  For inputs where
 * 4^k counters do not fit but x is small.  Output, capacities, ownership and
 * errors exactly as trial_hash (no positions or counts outputs); the candidate
 * list and member lists are identical to trial_hash's.  1 <= k <= min(l, 15),
 * n_trials <= 65535 and n_trials * x < 2^31 per call; ECAPACITY (with a
 * message) when a trial has more than 4096 enriched buckets. */
int trial_hash_allpairs(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l, int k,
                        int s, uint64_t seed, int64_t trial_begin, int64_t n_trials,
                        int64_t cap_cand, int64_t cap_members, int32_t *cand_trial_dev,
                        uint32_t *cand_key_dev, int32_t *cand_cnt_dev, int64_t *cand_off_dev,
                        int32_t *members_dev, int64_t *totals_dev, void *stream);

/* ---- the protein alphabet (Section 2, |Sigma| = 20) ---------------------- */

/* Algorithm 2 with Section 5.1's OOPS EM over the 20 amino-acid letters
 * ACDEFGHIKLMNPQRSTVWY (codes 0..19, either case; any other character returns
 * PROJ_EBADCHAR with its index in the message).  Host ASCII sequences in
 * linear form (ascii[seq_off[t]], seq_off[t+1], every length >= l, 1 <= l <=
 * 32).  k, s and m are required (the Section 5 formulas are stated for DNA):
 * 1 <= k <= min(l, 6) (keys base 20 = the projected residues read
 * most-significant first), s >= 1, 1 <= m <= 65535; trials draw their
 * positions as in trial_hash.  Enriched buckets come from a per-trial sort
 * of (key, l-mer) pairs in shared memory when x <= 16384, else from the
 * all-pairs comparison (trial_hash_allpairs' scheme, ECAPACITY above 4096
 * enriched buckets per trial); m * x < 2^31.  theta^0 and em_iters OOPS iterations:
 * scores and exponentials in FP32, M-step counts in 64-bit fixed point (2^-40),
 * log-likelihoods in FP64 (results do not depend on thread scheduling);
 * ranking, sites and Score as projection_find.  out->pwm holds [l][20] floats; out->win_key is
 * the base-20 key.  Copies in, computes, copies out, synchronises `stream`. */
int projection_find_protein(const uint8_t *ascii, const int64_t *seq_off, int t, int l, int k,
                            int s, int m, uint64_t seed, int em_iters, float pseudocount,
                            projection_result *out, void *stream);

/* ---- step 1 for a batch, on the device (Section 5) ---------------------- */

/* Algorithm 2 step 1 ("if not specified") for n instances held on the device:
 * k = l - d - 1, s = max(3, ceil(2x / 4^k)), m = ceil(log(1 - q) / log B) with
 * B = P[Binomial(t, p) < s] and p = C(l-d, k) / C(l, k) (Section 5), each only
 * where the caller's entry is 0 (nonzero entries are kept).  All arrays are
 * device int32 [n] except x_dev (int64 [n], l-mers of each instance); k, s and
 * m are read and written in place.  status_dev[i]: 0 OK, -1 invalid instance
 * (t < 1, l outside 1..32, d outside 0..l-1, k outside 1..l), -2 no finite
 * trial count (k > l - d, or m above 2^24; m is then 0).  The same formulas as
 * projection_default_params, evaluated in FP64 on the GPU.  Asynchronous on
 * `stream`; EINVAL for n < 0, q outside (0, 1) or NULL arrays. */
int projection_params_batch(int n, const int32_t *t_dev, const int64_t *x_dev,
                            const int32_t *l_dev, const int32_t *d_dev, int32_t *k_dev,
                            int32_t *s_dev, int32_t *m_dev, int32_t *status_dev, double q,
                            void *stream);

/* ---- failure detection --------------------------------------------------- */

/* Self-test of the bounded waits used by the tensor-core kernels: launches a
 * kernel that waits on an mbarrier nothing arrives on, with a limit of
 * timeout_ns (<= 2 s) measured on the GPU's global timer.  Returns
 * PROJ_ETIMEOUT when the wait expired and the kernel returned (the expected
 * outcome; the CUDA context stays usable), PROJ_ECUDA otherwise.
 * Synchronises `stream`. */
int projection_selftest_wait(int64_t timeout_ns, void *stream);

/* ---- measurement helper (no counterpart in the paper) -------------------- */

/* The shared-memory histogram rate that the bucket kernels (Algorithm 2 steps
 * 2b-2c) are measured against: one 1024-thread CTA per SM counts
 * register-generated pseudo-random keys into a shared-memory histogram laid out
 * as the bucket kernels lay out 4^k buckets (u32 counters up to 128 KB, else
 * u16 pairs over 65,536 buckets).  *updates_per_s = increments per second,
 * whole GPU (fastest of three timed launches after one warm-up).  k in 1..10.
 * Synchronises `stream`. */
int projection_hist_peak(int k, double *updates_per_s, void *stream);

/* The GPU's exp2 rate (ex2.approx, the EM kernels' one exponential per score)
 * measured with independent dependency chains on every SM: *ex2_per_s =
 * exponentials per second (best of 3 timed launches after a warm-up).
 * Synchronises `stream`. */
int projection_ex2_peak(double *ex2_per_s, void *stream);

/* ---- tracing (CUDA-event timers per kernel) ----------------------------- */

/* on != 0: start recording a CUDA event pair around every kernel the library
 * launches (on the stream it launches on) and clear earlier records; on == 0:
 * stop recording.  Off by default; costs two event records per launch. */
int projection_trace_enable(int on);

/* Sums the records of kernels whose name starts with `prefix` ("" = all):
 * *total_ms = summed device time, *launches = number of launches.  Waits for
 * the recorded events.  Kernel names: pack, background, positions, params,
 * hash_partition, hash_count, hash_scan, hash_fill, hash_table, select,
 * hash_gather, allpairs, enrich_sort, theta0, em_xtiles, em_tc, em_fp32,
 * em_reduce, cand_sites, finalize (protein searches record under the same names). */
int projection_trace_read(const char *prefix, double *total_ms, int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* PROJECTION_H */
