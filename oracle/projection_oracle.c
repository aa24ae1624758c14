/*
 * projection_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow CPU statement of the PROJECTION motif finder as restated in
 * Clemente, Cabarle & Adorna, "PROJECTION Algorithm for Motif Finding on GPUs"
 * (arXiv 1605.06904): the random projection and hashing of Algorithm 2
 * (Section 5), the parameter choice of Section 5 (k, s and the trial bound m),
 * the enriched-bucket rule of Section 6, and the EM refinement of Section 5.1.
 * Floating point is IEEE double throughout.
 *
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
 * load the library built from this file.  It shares no code, header, table or
 * helper with the CUDA library: the two are compared, never combined.
 *
 * Readings of the paper where it is silent or garbled (each restated where it
 * is used):
 *   R1  codes: A=0, C=1, T=2, G=3 (Section 6, base-|Sigma| hashing); any other
 *       character is rejected.
 *   R2  Algorithm 2 step 2a draws "(l-k) random numbers in [0,l]": read as l-k
 *       DISTINCT excluded positions in {0..l-1}, drawn by a partial
 *       Fisher-Yates shuffle fed by Philox4x32-10 (Salmon et al., SC'11) keyed
 *       by the seed with counter (trial, block); the k kept positions are the
 *       complement in increasing order ("order preserved", Section 5).
 *   R3  a bucket is enriched when it holds at least s l-mers; one candidate per
 *       (trial, key); l-mers never span two sequences.
 *   R4  background = 0-order base frequencies of the whole input, held fixed
 *       during EM; a base absent from the input counts as one occurrence.
 *   R5  EM is the one-occurrence-per-sequence (OOPS) model with a uniform prior
 *       over sites and a pseudocount beta per base in the M-step.
 *   R15 the zero-or-one-occurrence (ZOOPS) model named in Section 2 is read as
 *       the standard two-component mixture with a fixed site probability gamma
 *       per sequence (uniform over its starts) and the MAP M-step whose
 *       denominator is the expected number of sites plus 4 beta.
 *
 * Parity status: every function below is pinned by a CPU test (worked example
 * of Figures 1, 2 and 4, Philox known-answer vectors, brute-force bucket
 * enumeration, closed-form EM special cases, the non-decreasing MAP objective,
 * and planted-motif recovery) except where its header says "parity unpinned".
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* R1: alphabet codes (Section 6: A:0, C:1, T:2, G:3).                        */
/* ------------------------------------------------------------------------- */

/* Returns -1 when every character is one of ACGT/acgt, else the index of the
 * first character that is not. */
int64_t orc_encode(const uint8_t *ascii, int64_t n, uint8_t *codes) {
    for (int64_t i = 0; i < n; ++i) {
        switch (ascii[i]) {
        case 'A': case 'a': codes[i] = 0; break;
        case 'C': case 'c': codes[i] = 1; break;
        case 'T': case 't': codes[i] = 2; break;
        case 'G': case 'g': codes[i] = 3; break;
        default: return i;
        }
    }
    return -1;
}

/* Linear 2-bit form of the input (Section 6: the inputs are passed in linear
 * form): base b sits in word b/16 at bits 2*(b%16) .. 2*(b%16)+1.  Unused high
 * bits of the last word are zero. */
void orc_pack2(const uint8_t *codes, int64_t n, uint32_t *words) {
    int64_t nw = (n + 15) / 16;
    for (int64_t w = 0; w < nw; ++w) words[w] = 0;
    for (int64_t b = 0; b < n; ++b)
        words[b / 16] |= (uint32_t)(codes[b] & 3u) << (2 * (b % 16));
}

/* ------------------------------------------------------------------------- */
/* R2: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its    */
/* published definition: 10 rounds of two 32x32->64 multiplies with the      */
/* Weyl-sequence key schedule.                                                */
/* ------------------------------------------------------------------------- */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u; /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u; /* key increments */
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Algorithm 2 step 2a with reading R2.  Writes the k projected positions
 * (0-based, increasing) to pos[0..k-1].  Returns 0, or -1 on bad l/k. */
int orc_positions(uint64_t seed, uint64_t trial, int l, int k, int32_t *pos) {
    if (l < 1 || l > 32 || k < 1 || k > l) return -1;
    int perm[32];
    for (int i = 0; i < l; ++i) perm[i] = i;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t words[4];
    int excluded = l - k;
    for (int i = 0; i < excluded; ++i) {
        if (i % 4 == 0) {
            uint32_t ctr[4] = {(uint32_t)trial, (uint32_t)(i / 4), (uint32_t)(trial >> 32), 0u};
            orc_philox4x32_10(ctr, key, words);
        }
        uint32_t u = words[i % 4];
        /* j uniform in [i, l): floor(u * (l - i) / 2^32) */
        int j = i + (int)(((uint64_t)u * (uint64_t)(l - i)) >> 32);
        int tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
    }
    int is_excluded[32] = {0};
    for (int i = 0; i < excluded; ++i) is_excluded[perm[i]] = 1;
    int q = 0;
    for (int p = 0; p < l; ++p)
        if (!is_excluded[p]) pos[q++] = p;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* l-mers, projection h_k and base-4 hashing (Section 5 Algorithm 2 steps    */
/* 2b-2c; Section 6, most significant digit first).                           */
/* ------------------------------------------------------------------------- */

/* seq_off[i]..seq_off[i+1] delimit sequence i in the concatenated codes.
 * lmer_off[i] = number of l-mers in sequences 0..i-1 (the global l-mer id of
 * S_{i,0}); a sequence shorter than l contributes none.  Returns x. */
int64_t orc_lmer_offsets(const int64_t *seq_off, int t, int l, int64_t *lmer_off) {
    lmer_off[0] = 0;
    for (int i = 0; i < t; ++i) {
        int64_t n = seq_off[i + 1] - seq_off[i];
        int64_t c = n >= l ? n - l + 1 : 0;
        lmer_off[i + 1] = lmer_off[i] + c;
    }
    return lmer_off[t];
}

/* key of every l-mer, in global l-mer order (sequence-major, start ascending):
 * key = sum_q code(S_i[j + pos_q]) * 4^(k-1-q). */
void orc_keys(const uint8_t *codes, const int64_t *seq_off, int t, int l, int k,
              const int32_t *pos, uint32_t *keys) {
    int64_t g = 0;
    for (int i = 0; i < t; ++i) {
        int64_t n = seq_off[i + 1] - seq_off[i];
        for (int64_t j = 0; j + l <= n; ++j) {
            const uint8_t *lmer = codes + seq_off[i] + j;
            uint32_t key = 0;
            for (int q = 0; q < k; ++q) key = key * 4u + lmer[pos[q]];
            keys[g++] = key;
        }
    }
}

/* Algorithm 2 step 2c: bucket sizes over the |Sigma|^k = 4^k bins. */
void orc_counts(const uint32_t *keys, int64_t x, int k, uint32_t *counts) {
    uint64_t nb = (uint64_t)1 << (2 * k);
    for (uint64_t b = 0; b < nb; ++b) counts[b] = 0;
    for (int64_t g = 0; g < x; ++g) counts[keys[g]] += 1;
}

typedef struct { uint32_t key; int32_t id; } orc_pair;

static int cmp_pair(const void *a, const void *b) {
    const orc_pair *p = (const orc_pair *)a, *q = (const orc_pair *)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return (p->id > q->id) - (p->id < q->id);
}

/* Algorithm 2 step 3 with reading R3, for ONE trial: the buckets holding at
 * least s l-mers, ascending by key, each with its members (global l-mer ids,
 * ascending).  The grouping is a sort of (key, id) pairs.  Writes at most
 * cap_c candidates and cap_m members; always returns the full candidate count
 * and stores the full member count in *n_members. */
int64_t orc_enriched(const uint32_t *keys, int64_t x, int s,
                     uint32_t *cand_key, int32_t *cand_cnt, int64_t *cand_off,
                     int32_t *members, int64_t cap_c, int64_t cap_m, int64_t *n_members) {
    orc_pair *pairs = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)(x > 0 ? x : 1));
    for (int64_t g = 0; g < x; ++g) { pairs[g].key = keys[g]; pairs[g].id = (int32_t)g; }
    qsort(pairs, (size_t)x, sizeof(orc_pair), cmp_pair);
    int64_t nc = 0, nm = 0;
    int64_t a = 0;
    while (a < x) {
        int64_t b = a;
        while (b < x && pairs[b].key == pairs[a].key) ++b;
        int64_t cnt = b - a;
        if (cnt >= s) {
            if (nc < cap_c) {
                cand_key[nc] = pairs[a].key;
                cand_cnt[nc] = (int32_t)cnt;
                cand_off[nc] = nm;
            }
            for (int64_t e = a; e < b; ++e) {
                if (nm < cap_m) members[nm] = pairs[e].id;
                ++nm;
            }
            ++nc;
        }
        a = b;
    }
    free(pairs);
    *n_members = nm;
    return nc;
}

/* ------------------------------------------------------------------------- */
/* Section 5 parameter choice.                                                */
/* ------------------------------------------------------------------------- */

static double log_choose(int n, int r) {
    if (r < 0 || r > n) return -INFINITY;
    return lgamma(n + 1.0) - lgamma(r + 1.0) - lgamma(n - r + 1.0);
}

/* m = ceil( log(1-q) / log B_{t_hat, p_hat}(s) ), p_hat = C(l-d, k) / C(l, k),
 * B(s) = P[Binomial(t_hat, p_hat) < s].  Returns -1 when no finite m exists
 * (p_hat = 0, i.e. k > l-d, or q outside (0,1)). */
int64_t orc_m_bound(int l, int d, int k, int s, int t_hat, double q) {
    if (k > l - d || k < 1 || q <= 0.0 || q >= 1.0 || t_hat < 1 || s < 1) return -1;
    double p = exp(log_choose(l - d, k) - log_choose(l, k));
    double B = 0.0;
    for (int c = 0; c < s && c <= t_hat; ++c)
        B += exp(log_choose(t_hat, c) + c * log(p) + (t_hat - c) * log1p(-p));
    if (B >= 1.0) return -1;
    if (B <= 0.0) return 1;
    return (int64_t)ceil(log(1.0 - q) / log(B));
}

/* ------------------------------------------------------------------------- */
/* Section 5.1: motif model theta (4 x (l+1): column 0 background, columns    */
/* 1..l the PWM; stored here as the background bg[4] and pwm[l][4]).         */
/* ------------------------------------------------------------------------- */

/* R4: background frequencies of the whole input. */
void orc_background(const uint8_t *codes, int64_t n, double bg[4]) {
    int64_t c[4] = {0, 0, 0, 0};
    for (int64_t b = 0; b < n; ++b) c[codes[b]] += 1;
    int64_t tot = 0;
    for (int a = 0; a < 4; ++a) { if (c[a] == 0) c[a] = 1; tot += c[a]; }
    for (int a = 0; a < 4; ++a) bg[a] = (double)c[a] / (double)tot;
}

/* Maps a global l-mer id to its sequence i and start j. */
static void lmer_locate(const int64_t *lmer_off, int t, int64_t g, int *i_out, int64_t *j_out) {
    int lo = 0, hi = t - 1;
    while (lo < hi) { /* last i with lmer_off[i] <= g */
        int mid = (lo + hi + 1) / 2;
        if (lmer_off[mid] <= g) lo = mid; else hi = mid - 1;
    }
    *i_out = lo;
    *j_out = g - lmer_off[lo];
}

/* theta^0 of Example 1 / Figure 4: column frequencies of the bucket's l-mers,
 * (count_a(p) + beta) / (cnt + 4 beta).  With beta = 0 this is the profile
 * P(s) of Figure 2 divided by the bucket size. */
void orc_theta0(const uint8_t *codes, const int64_t *seq_off, const int64_t *lmer_off, int t,
                int l, const int32_t *members, int cnt, double beta, double *pwm) {
    double n[32][4];
    memset(n, 0, sizeof n);
    for (int e = 0; e < cnt; ++e) {
        int i; int64_t j;
        lmer_locate(lmer_off, t, members[e], &i, &j);
        const uint8_t *lmer = codes + seq_off[i] + j;
        for (int p = 0; p < l; ++p) n[p][lmer[p]] += 1.0;
    }
    for (int p = 0; p < l; ++p)
        for (int a = 0; a < 4; ++a) pwm[p * 4 + a] = (n[p][a] + beta) / ((double)cnt + 4.0 * beta);
}

/* r(i,j) = sum_p [log pwm_p(x_{i,j+p}) - log bg(x_{i,j+p})] for all starts j of
 * sequence i; returns the number of starts. */
static int64_t seq_scores(const uint8_t *codes, const int64_t *seq_off, int i, int l,
                          const double W[32][4], double *r) {
    int64_t n = seq_off[i + 1] - seq_off[i];
    int64_t ns = n >= l ? n - l + 1 : 0;
    for (int64_t j = 0; j < ns; ++j) {
        const uint8_t *lmer = codes + seq_off[i] + j;
        double acc = 0.0;
        for (int p = 0; p < l; ++p) acc += W[p][lmer[p]];
        r[j] = acc;
    }
    return ns;
}

static void log_ratio(const double *pwm, const double bg[4], int l, double W[32][4]) {
    for (int p = 0; p < l; ++p)
        for (int a = 0; a < 4; ++a) W[p][a] = log(pwm[p * 4 + a]) - log(bg[a]);
}

/* OOPS EM for ONE starting model (reading R5).  E-step: per sequence i the
 * posterior over starts z(i,j) = exp(r(i,j)) / sum_j' exp(r(i,j')); the
 * log-likelihood ratio against the all-background model is
 *     LL = sum_i [ log sum_j exp r(i,j) - log(n_i - l + 1) ].
 * M-step: pwm_p(a) = (sum_{i,j} z(i,j) [x_{i,j+p} = a] + beta) / (t' + 4 beta),
 * t' = number of sequences holding at least one l-mer.
 * Runs E, M, E, M, ... : `iters` M-steps, then a final E-step.  On return pwm
 * holds the model after `iters` M-steps, *ll its log-likelihood ratio,
 * lse[i] (optional) the per-sequence log-sum-exp, trace[0..iters] (optional)
 * the LL of each E-step. */
static void em_one(const uint8_t *codes, const int64_t *seq_off, int t, int l, const double bg[4],
                   double *pwm, int iters, double beta, double *ll, double *lse, double *trace,
                   double *r) {
    double W[32][4];
    int tprime = 0;
    for (int i = 0; i < t; ++i)
        if (seq_off[i + 1] - seq_off[i] >= l) ++tprime;
    for (int it = 0; it <= iters; ++it) {
        log_ratio(pwm, bg, l, W);
        double N[32][4];
        memset(N, 0, sizeof N);
        double LL = 0.0;
        for (int i = 0; i < t; ++i) {
            int64_t ns = seq_scores(codes, seq_off, i, l, W, r);
            if (ns == 0) { if (lse && it == iters) lse[i] = 0.0; continue; }
            double mx = r[0];
            for (int64_t j = 1; j < ns; ++j) if (r[j] > mx) mx = r[j];
            double S = 0.0;
            for (int64_t j = 0; j < ns; ++j) S += exp(r[j] - mx);
            double L = mx + log(S);
            LL += L - log((double)ns);
            if (lse && it == iters) lse[i] = L;
            if (it < iters) {
                for (int64_t j = 0; j < ns; ++j) {
                    double z = exp(r[j] - L);
                    const uint8_t *lmer = codes + seq_off[i] + j;
                    for (int p = 0; p < l; ++p) N[p][lmer[p]] += z;
                }
            }
        }
        if (trace) trace[it] = LL;
        if (it == iters) { *ll = LL; break; }
        for (int p = 0; p < l; ++p)
            for (int a = 0; a < 4; ++a) pwm[p * 4 + a] = (N[p][a] + beta) / ((double)tprime + 4.0 * beta);
    }
}

/* ZOOPS EM for ONE starting model (zero or one occurrence per sequence, the
 * second search model of Section 2; reading R15).  A sequence holds one site
 * with prior probability gamma (fixed), uniform over its n_i - l + 1 starts,
 * or no site.  E-step, per sequence i with ns_i starts:
 *     L_i = log[ (1 - gamma) + (gamma / ns_i) sum_j exp r(i,j) ]
 * (log-likelihood ratio against the all-background model), and the posterior
 * of a site at j
 *     z(i,j) = (gamma / ns_i) exp r(i,j) / exp(L_i).
 * M-step: pwm_p(a) = (sum_{i,j} z(i,j) [x_{i,j+p} = a] + beta)
 *                    / (sum_{i,j} z(i,j) + 4 beta).
 * LL = sum_i L_i.  gamma = 1 is the OOPS model (up to rounding).  Same
 * iteration order as em_one. */
static double log_add(double a, double b) {
    double hi = a > b ? a : b, lo = a > b ? b : a;
    if (hi == -INFINITY) return -INFINITY;
    return hi + log1p(exp(lo - hi));
}

static void em_one_zoops(const uint8_t *codes, const int64_t *seq_off, int t, int l,
                         const double bg[4], double *pwm, int iters, double beta, double gamma,
                         double *ll, double *trace, double *r) {
    double W[32][4];
    const double log_no = gamma < 1.0 ? log1p(-gamma) : -INFINITY;
    for (int it = 0; it <= iters; ++it) {
        log_ratio(pwm, bg, l, W);
        double N[32][4];
        memset(N, 0, sizeof N);
        double LL = 0.0, Z = 0.0;
        for (int i = 0; i < t; ++i) {
            int64_t ns = seq_scores(codes, seq_off, i, l, W, r);
            if (ns == 0) continue;
            double mx = r[0];
            for (int64_t j = 1; j < ns; ++j) if (r[j] > mx) mx = r[j];
            double S = 0.0;
            for (int64_t j = 0; j < ns; ++j) S += exp(r[j] - mx);
            const double log_site = log(gamma / (double)ns) + mx + log(S);
            const double L = log_add(log_no, log_site);
            LL += L;
            if (it < iters) {
                for (int64_t j = 0; j < ns; ++j) {
                    double z = exp(log(gamma / (double)ns) + r[j] - L);
                    const uint8_t *lmer = codes + seq_off[i] + j;
                    for (int p = 0; p < l; ++p) N[p][lmer[p]] += z;
                    Z += z;
                }
            }
        }
        if (trace) trace[it] = LL;
        if (it == iters) { *ll = LL; break; }
        for (int p = 0; p < l; ++p)
            for (int a = 0; a < 4; ++a) pwm[p * 4 + a] = (N[p][a] + beta) / (Z + 4.0 * beta);
    }
}

typedef struct {
    const uint8_t *codes; const int64_t *seq_off; int t, l; const double *bg;
    double *pwm; int64_t C; int iters; double beta; double *ll, *lse, *trace;
    int64_t c_begin, c_end; int64_t max_ns;
    double gamma;  /* > 0 and < 1: ZOOPS with this site probability; else OOPS */
} em_job;

static void *em_worker(void *arg) {
    em_job *jb = (em_job *)arg;
    double *r = (double *)malloc(sizeof(double) * (size_t)(jb->max_ns > 0 ? jb->max_ns : 1));
    for (int64_t c = jb->c_begin; c < jb->c_end; ++c) {
        if (jb->gamma > 0.0)
            em_one_zoops(jb->codes, jb->seq_off, jb->t, jb->l, jb->bg, jb->pwm + c * jb->l * 4,
                         jb->iters, jb->beta, jb->gamma, jb->ll + c,
                         jb->trace ? jb->trace + c * (jb->iters + 1) : NULL, r);
        else
            em_one(jb->codes, jb->seq_off, jb->t, jb->l, jb->bg, jb->pwm + c * jb->l * 4, jb->iters,
                   jb->beta, jb->ll + c, jb->lse ? jb->lse + c * jb->t : NULL,
                   jb->trace ? jb->trace + c * (jb->iters + 1) : NULL, r);
    }
    free(r);
    return NULL;
}

/* EM for C independent starting models pwm[C][l][4] (refined in place).
 * Candidates are independent, so they are split across `nthreads` threads;
 * the arithmetic of each candidate is the same as with one thread. */
static int em_run(const uint8_t *codes, const int64_t *seq_off, int t, int l, const double bg[4],
                  double *pwm, int64_t C, int iters, double beta, double gamma, double *ll,
                  double *lse, double *trace, int nthreads) {
    if (l < 1 || l > 32 || iters < 0 || t < 1) return -1;
    int64_t max_ns = 0;
    for (int i = 0; i < t; ++i) {
        int64_t n = seq_off[i + 1] - seq_off[i];
        if (n - l + 1 > max_ns) max_ns = n - l + 1;
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > C) nthreads = C > 0 ? (int)C : 1;
    em_job *jobs = (em_job *)calloc((size_t)nthreads, sizeof(em_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int w = 0; w < nthreads; ++w) {
        em_job *jb = &jobs[w];
        jb->codes = codes; jb->seq_off = seq_off; jb->t = t; jb->l = l; jb->bg = bg;
        jb->pwm = pwm; jb->C = C; jb->iters = iters; jb->beta = beta; jb->ll = ll;
        jb->lse = lse; jb->trace = trace; jb->max_ns = max_ns; jb->gamma = gamma;
        jb->c_begin = C * w / nthreads; jb->c_end = C * (w + 1) / nthreads;
    }
    for (int w = 1; w < nthreads; ++w) pthread_create(&th[w], NULL, em_worker, &jobs[w]);
    em_worker(&jobs[0]);
    for (int w = 1; w < nthreads; ++w) pthread_join(th[w], NULL);
    free(jobs); free(th);
    return 0;
}

int orc_em(const uint8_t *codes, const int64_t *seq_off, int t, int l, const double bg[4],
           double *pwm, int64_t C, int iters, double beta, double *ll, double *lse,
           double *trace, int nthreads) {
    return em_run(codes, seq_off, t, l, bg, pwm, C, iters, beta, 0.0, ll, lse, trace, nthreads);
}

/* ZOOPS EM (em_one_zoops) for C starting models; 0 < gamma <= 1. */
int orc_em_zoops(const uint8_t *codes, const int64_t *seq_off, int t, int l, const double bg[4],
                 double *pwm, int64_t C, int iters, double beta, double gamma, double *ll,
                 double *trace, int nthreads) {
    if (!(gamma > 0.0 && gamma <= 1.0)) return -1;
    return em_run(codes, seq_off, t, l, bg, pwm, C, iters, beta, gamma, ll, NULL, trace, nthreads);
}

/* Predicted sites: for each sequence the first start maximising r(i,j)
 * (equivalently the posterior z(i,j)); -1 for a sequence without l-mers. */
void orc_sites(const uint8_t *codes, const int64_t *seq_off, int t, int l, const double bg[4],
               const double *pwm, int32_t *sites) {
    double W[32][4];
    log_ratio(pwm, bg, l, W);
    int64_t max_ns = 1;
    for (int i = 0; i < t; ++i) {
        int64_t n = seq_off[i + 1] - seq_off[i];
        if (n - l + 1 > max_ns) max_ns = n - l + 1;
    }
    double *r = (double *)malloc(sizeof(double) * (size_t)max_ns);
    for (int i = 0; i < t; ++i) {
        int64_t ns = seq_scores(codes, seq_off, i, l, W, r);
        int64_t best = ns > 0 ? 0 : -1;
        for (int64_t j = 1; j < ns; ++j) if (r[j] > r[best]) best = j;
        sites[i] = (int32_t)best;
    }
    free(r);
}

/* Consensus string of Section 2: per column the base of largest weight; the
 * paper leaves ties arbitrary, here the lowest code (A, C, T, G order) wins.
 * Writes l letters and a terminating NUL. */
void orc_consensus(const double *pwm, int l, char *out) {
    static const char letter[4] = {'A', 'C', 'T', 'G'};
    for (int p = 0; p < l; ++p) {
        int best = 0;
        for (int a = 1; a < 4; ++a) if (pwm[p * 4 + a] > pwm[p * 4 + best]) best = a;
        out[p] = letter[best];
    }
    out[l] = 0;
}

/* Score(s, DNA) of Section 2: sum over the l columns of the alignment A(s) of
 * the largest base count.  Sequences whose site is -1 are left out. */
int orc_score(const uint8_t *codes, const int64_t *seq_off, int t, int l, const int32_t *sites) {
    int total = 0;
    for (int p = 0; p < l; ++p) {
        int c[4] = {0, 0, 0, 0};
        for (int i = 0; i < t; ++i) {
            if (sites[i] < 0) continue;
            c[codes[seq_off[i] + sites[i] + p]] += 1;
        }
        int m = c[0];
        for (int a = 1; a < 4; ++a) if (c[a] > m) m = c[a];
        total += m;
    }
    return total;
}

/* ------------------------------------------------------------------------- */
/* R17: the protein alphabet.  Section 2 takes Sigma = {A, C, G, T} for DNA and */
/* |Sigma| = 20 for proteins; read here as the 20 amino-acid letters           */
/* ACDEFGHIKLMNPQRSTVWY with codes 0..19 in that order (upper or lower case).  */
/* The functions below are the DNA ones with the alphabet size A as a          */
/* parameter (keys base A, most significant position first; models A x l).    */
/* With A = 4 and codes 0..3 they compute exactly what the DNA functions do.   */
/* ------------------------------------------------------------------------- */

int64_t orc_encode_aa(const uint8_t *ascii, int64_t n, uint8_t *codes) {
    static const char letters[] = "ACDEFGHIKLMNPQRSTVWY";
    for (int64_t i = 0; i < n; ++i) {
        int c = ascii[i];
        if (c >= 'a' && c <= 'z') c -= 32;
        int code = -1;
        for (int a = 0; a < 20; ++a) if (letters[a] == c) { code = a; break; }
        if (code < 0) return i;
        codes[i] = (uint8_t)code;
    }
    return -1;
}

void orc_keys_a(const uint8_t *codes, const int64_t *seq_off, int t, int l, int k,
                const int32_t *pos, int A, uint32_t *keys) {
    int64_t g = 0;
    for (int i = 0; i < t; ++i) {
        int64_t n = seq_off[i + 1] - seq_off[i];
        for (int64_t j = 0; j + l <= n; ++j) {
            const uint8_t *lmer = codes + seq_off[i] + j;
            uint32_t key = 0;
            for (int q = 0; q < k; ++q) key = key * (uint32_t)A + lmer[pos[q]];
            keys[g++] = key;
        }
    }
}

void orc_background_a(const uint8_t *codes, int64_t n, int A, double *bg) {
    int64_t c[32] = {0};
    for (int64_t b = 0; b < n; ++b) c[codes[b]] += 1;
    int64_t tot = 0;
    for (int a = 0; a < A; ++a) { if (c[a] == 0) c[a] = 1; tot += c[a]; }
    for (int a = 0; a < A; ++a) bg[a] = (double)c[a] / (double)tot;
}

void orc_theta0_a(const uint8_t *codes, const int64_t *seq_off, const int64_t *lmer_off, int t,
                  int l, const int32_t *members, int cnt, double beta, int A, double *pwm) {
    double n[32][32];
    memset(n, 0, sizeof n);
    for (int e = 0; e < cnt; ++e) {
        int i;
        int64_t j;
        lmer_locate(lmer_off, t, members[e], &i, &j);
        const uint8_t *lmer = codes + seq_off[i] + j;
        for (int p = 0; p < l; ++p) n[p][lmer[p]] += 1.0;
    }
    for (int p = 0; p < l; ++p)
        for (int a = 0; a < A; ++a) pwm[p * A + a] = (n[p][a] + beta) / ((double)cnt + A * beta);
}

/* OOPS EM (as em_one) over an alphabet of A letters: r(i,j) = sum_p
 * [log pwm_p(x) - log bg(x)], z = softmax over the starts, LL = sum_i [log
 * sum_j e^r - log ns_i], pwm_p(a) = (sum z [x = a] + beta) / (t' + A beta). */
static void em_one_a(const uint8_t *codes, const int64_t *seq_off, int t, int l, int A,
                     const double *bg, double *pwm, int iters, double beta, double *ll,
                     double *r) {
    double W[32][32];
    int tprime = 0;
    for (int i = 0; i < t; ++i)
        if (seq_off[i + 1] - seq_off[i] >= l) ++tprime;
    for (int it = 0; it <= iters; ++it) {
        for (int p = 0; p < l; ++p)
            for (int a = 0; a < A; ++a) W[p][a] = log(pwm[p * A + a]) - log(bg[a]);
        double N[32][32];
        memset(N, 0, sizeof N);
        double LL = 0.0;
        for (int i = 0; i < t; ++i) {
            int64_t n = seq_off[i + 1] - seq_off[i];
            int64_t ns = n >= l ? n - l + 1 : 0;
            if (ns == 0) continue;
            for (int64_t j = 0; j < ns; ++j) {
                const uint8_t *lmer = codes + seq_off[i] + j;
                double acc = 0.0;
                for (int p = 0; p < l; ++p) acc += W[p][lmer[p]];
                r[j] = acc;
            }
            double mx = r[0];
            for (int64_t j = 1; j < ns; ++j) if (r[j] > mx) mx = r[j];
            double S = 0.0;
            for (int64_t j = 0; j < ns; ++j) S += exp(r[j] - mx);
            double L = mx + log(S);
            LL += L - log((double)ns);
            if (it < iters) {
                for (int64_t j = 0; j < ns; ++j) {
                    double z = exp(r[j] - L);
                    const uint8_t *lmer = codes + seq_off[i] + j;
                    for (int p = 0; p < l; ++p) N[p][lmer[p]] += z;
                }
            }
        }
        if (it == iters) { *ll = LL; break; }
        for (int p = 0; p < l; ++p)
            for (int a = 0; a < A; ++a)
                pwm[p * A + a] = (N[p][a] + beta) / ((double)tprime + A * beta);
    }
}

typedef struct {
    const uint8_t *codes; const int64_t *seq_off; int t, l, A; const double *bg;
    double *pwm; int iters; double beta; double *ll; int64_t c_begin, c_end, max_ns;
} em_a_job;

static void *em_a_worker(void *arg) {
    em_a_job *jb = (em_a_job *)arg;
    double *r = (double *)malloc(sizeof(double) * (size_t)(jb->max_ns > 0 ? jb->max_ns : 1));
    for (int64_t c = jb->c_begin; c < jb->c_end; ++c)
        em_one_a(jb->codes, jb->seq_off, jb->t, jb->l, jb->A, jb->bg,
                 jb->pwm + c * jb->l * jb->A, jb->iters, jb->beta, jb->ll + c, r);
    free(r);
    return NULL;
}

int orc_em_a(const uint8_t *codes, const int64_t *seq_off, int t, int l, int A, const double *bg,
             double *pwm, int64_t C, int iters, double beta, double *ll, int nthreads) {
    if (l < 1 || l > 32 || A < 2 || A > 32 || iters < 0 || t < 1) return -1;
    int64_t max_ns = 0;
    for (int i = 0; i < t; ++i) {
        int64_t n = seq_off[i + 1] - seq_off[i];
        if (n - l + 1 > max_ns) max_ns = n - l + 1;
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > C) nthreads = C > 0 ? (int)C : 1;
    em_a_job *jobs = (em_a_job *)calloc((size_t)nthreads, sizeof(em_a_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int w = 0; w < nthreads; ++w) {
        em_a_job *jb = &jobs[w];
        jb->codes = codes; jb->seq_off = seq_off; jb->t = t; jb->l = l; jb->A = A; jb->bg = bg;
        jb->pwm = pwm; jb->iters = iters; jb->beta = beta; jb->ll = ll; jb->max_ns = max_ns;
        jb->c_begin = C * w / nthreads; jb->c_end = C * (w + 1) / nthreads;
    }
    for (int w = 1; w < nthreads; ++w) pthread_create(&th[w], NULL, em_a_worker, &jobs[w]);
    em_a_worker(&jobs[0]);
    for (int w = 1; w < nthreads; ++w) pthread_join(th[w], NULL);
    free(jobs); free(th);
    return 0;
}

void orc_sites_a(const uint8_t *codes, const int64_t *seq_off, int t, int l, int A,
                 const double *bg, const double *pwm, int32_t *sites) {
    double W[32][32];
    for (int p = 0; p < l; ++p)
        for (int a = 0; a < A; ++a) W[p][a] = log(pwm[p * A + a]) - log(bg[a]);
    for (int i = 0; i < t; ++i) {
        int64_t n = seq_off[i + 1] - seq_off[i];
        int64_t ns = n >= l ? n - l + 1 : 0, best = ns > 0 ? 0 : -1;
        double bv = -INFINITY;
        for (int64_t j = 0; j < ns; ++j) {
            const uint8_t *lmer = codes + seq_off[i] + j;
            double acc = 0.0;
            for (int p = 0; p < l; ++p) acc += W[p][lmer[p]];
            if (acc > bv) { bv = acc; best = j; }
        }
        sites[i] = (int32_t)best;
    }
}

/* Consensus over A letters: per column the letter of largest weight, ties to
 * the lowest code (R13); `letters` maps codes to characters. */
void orc_consensus_a(const double *pwm, int l, int A, const char *letters, char *out) {
    for (int p = 0; p < l; ++p) {
        int best = 0;
        for (int a = 1; a < A; ++a) if (pwm[p * A + a] > pwm[p * A + best]) best = a;
        out[p] = letters[best];
    }
    out[l] = 0;
}

int orc_score_a(const uint8_t *codes, const int64_t *seq_off, int t, int l, int A,
                const int32_t *sites) {
    int total = 0;
    for (int p = 0; p < l; ++p) {
        int c[32] = {0};
        for (int i = 0; i < t; ++i) {
            if (sites[i] < 0) continue;
            c[codes[seq_off[i] + sites[i] + p]] += 1;
        }
        int m = 0;
        for (int a = 0; a < A; ++a) if (c[a] > m) m = c[a];
        total += m;
    }
    return total;
}
