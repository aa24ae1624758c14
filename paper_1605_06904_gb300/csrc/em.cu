// Steps a6-a9: initial model theta^0 (Section 5.1, Example 1 / Figure 4),
// OOPS EM refinement of every enriched bucket (Section 5.1), and the FP64
// ranking and finalisation (Section 2's consensus and Score).
//
// FP32 path (PROJ_EM_FP32): one thread per candidate model; the threads of a
// CTA walk the same l-mers in lockstep, so the l-mer's codes are warp-uniform
// and the per-candidate tables W[4l][cand] and acc[4l][cand] in shared memory
// are read and written without bank conflicts.  Per sequence the posterior
// weights are accumulated against a running maximum (rescaled when it grows),
// then normalised by the sequence's sum: the E- and M-steps of one iteration
// read each l-mer once.  Sequences are split into G groups across CTAs when
// there are too few candidates to fill the GPU; partial sums are reduced in a
// fixed order, so results do not depend on timing.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace proj {

int run_em_tc(const uint32_t *packed, const Layout &L, const double *bg, const float *theta0,
              int64_t C, int iters, float beta, float *theta_out, double *ll, cudaStream_t st,
              double gamma, int *err_dev);

namespace {

constexpr int kEmThreads = 64;  // candidates per CTA in the FP32 path

// ---------------------------------------------------------------------------
// theta^0: column frequencies of the bucket's l-mers plus pseudocount.
// ---------------------------------------------------------------------------
__global__ void theta0_kernel(const uint32_t *__restrict__ packed, int64_t nwords,
                              const int32_t *__restrict__ seq_off,
                              const int32_t *__restrict__ lmer_off, int t, int l,
                              const int64_t *__restrict__ cand_off,
                              const int32_t *__restrict__ members, int64_t C, float beta,
                              float *__restrict__ theta0) {
    extern __shared__ float cnt[];  // [4l][blockDim]
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t c = blockIdx.x * (int64_t)nt + tid;
    const int L4 = 4 * l;
    for (int q = 0; q < L4; ++q) cnt[q * nt + tid] = 0.f;
    if (c >= C) return;
    const int64_t e0 = cand_off[c], e1 = cand_off[c + 1];
    for (int64_t e = e0; e < e1; ++e) {
        const int g = members[e];
        int lo = 0, hi = t - 1;  // last i with lmer_off[i] <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(lmer_off + mid) <= g) lo = mid; else hi = mid - 1;
        }
        const int64_t b0 = (int64_t)__ldg(seq_off + lo) + (g - __ldg(lmer_off + lo));
        const uint64_t win = window64(packed, nwords, b0);
        for (int p = 0; p < l; ++p) cnt[(p * 4 + (int)((win >> (2 * p)) & 3u)) * nt + tid] += 1.f;
    }
    const float den = (float)(e1 - e0) + 4.f * beta;
    for (int q = 0; q < L4; ++q) theta0[c * L4 + q] = (cnt[q * nt + tid] + beta) / den;
}

// theta0 with one warp per candidate, for searches that keep a few large
// buckets: the lanes split the bucket's members (each finds its sequence and
// window on its own) and count their bases in packed 8-bit counters, four
// codes of one position per register, folded across the warp after at most
// 255 members per lane.  The counts are integers, so the result is the same
// as the thread-per-candidate form's, bit for bit.
__global__ void __launch_bounds__(256) theta0_warp_kernel(
    const uint32_t *__restrict__ packed, int64_t nwords, const int32_t *__restrict__ seq_off,
    const int32_t *__restrict__ lmer_off, int t, int l, const int64_t *__restrict__ cand_off,
    const int32_t *__restrict__ members, int64_t C, float beta, float *__restrict__ theta0) {
    const int lane = threadIdx.x & 31;
    const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (c >= C) return;  // c is the same for the whole warp
    const int64_t e0 = cand_off[c], e1 = cand_off[c + 1];
    uint32_t tot[4] = {0u, 0u, 0u, 0u};  // lane q: entries q, q + 32, q + 64, q + 96
    for (int64_t base = e0; base < e1; base += 32 * 255) {
        uint32_t acc[32];
#pragma unroll
        for (int p = 0; p < 32; ++p) acc[p] = 0u;
        const int64_t end = min(e1, base + 32 * 255);
        for (int64_t e = base + lane; e < end; e += 32) {
            const int g = members[e];
            int lo = 0, hi = t - 1;  // last i with lmer_off[i] <= g
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(lmer_off + mid) <= g) lo = mid; else hi = mid - 1;
            }
            const int64_t b0 = (int64_t)__ldg(seq_off + lo) + (g - __ldg(lmer_off + lo));
            const uint64_t win = window64(packed, nwords, b0);
#pragma unroll
            for (int p = 0; p < 32; ++p) acc[p] += 1u << (((uint32_t)(win >> (2 * p)) & 3u) << 3);
        }
#pragma unroll
        for (int p = 0; p < 32; ++p) {
            if (p < l) {
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const uint32_t v = __reduce_add_sync(0xffffffffu, (acc[p] >> (8 * a)) & 255u);
                    if (lane == ((4 * p + a) & 31)) tot[(4 * p + a) >> 5] += v;
                }
            }
        }
    }
    const float den = (float)(e1 - e0) + 4.f * beta;
    const int L4 = 4 * l;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int q = 32 * r + lane;
        if (q < L4) theta0[c * L4 + q] = ((float)tot[r] + beta) / den;
    }
}

// ---------------------------------------------------------------------------
// One EM iteration (E-step + optional M-step) in FP32 for a tile of
// candidates and one group of sequences.
//
// Accuracy: the per-sequence sum S = sum_j exp(r - m) and the weighted counts
// acc[p][a] are compensated (Kahan) sums, exp is the accurate expf, and the
// per-sequence normalised counts and log-sum-exp are accumulated in FP64.
// Plain FP32 running sums over the ~10^3 l-mers of a sequence leave relative
// errors near n * 2^-24 in S, which the log-likelihood amplifies through the
// small PWM entries; compensation keeps it at a few ulp.
// ---------------------------------------------------------------------------
struct EmParams {
    const uint32_t *packed;
    int64_t nwords;
    const int32_t *seq_off;
    int t, l, G;
    const double *bg;
    const float *theta_in;
    double *part_acc;   // [G][C][4l] normalised counts of this group's sequences
    double *part_ll;    // [G][C]
    double *part_zs;    // [G][C] expected number of sites (ZOOPS)
    int64_t C;
    int mstep;
    double gamma;       // site probability per sequence: < 1 ZOOPS, 1 OOPS
};

// log(e^a + e^b) in FP64 (a may be -inf).
__device__ __forceinline__ double log_add_d(double a, double b) {
    const double hi = fmax(a, b), lo = fmin(a, b);
    return hi == -INFINITY ? -INFINITY : hi + log1p(exp(lo - hi));
}

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float v) {
    const float y = v - comp;
    const float s = sum + y;
    comp = (s - sum) - y;
    sum = s;
}

template <int LMAX>
__global__ void __launch_bounds__(kEmThreads) em_fp32_kernel(const EmParams P) {
    extern __shared__ float sm[];
    constexpr int NT = kEmThreads;
    const int tid = threadIdx.x;
    const int l = P.l, L4 = 4 * l;
    float *Ws = sm;                 // [4l][NT]
    float *acc = sm + L4 * NT;      // [4l][NT]
    float *cmp = sm + 2 * L4 * NT;  // [4l][NT] Kahan compensation of acc
    const int64_t c = blockIdx.x * (int64_t)NT + tid;
    const bool valid = c < P.C;
    const int g = blockIdx.y;
    double *tot = P.part_acc + ((int64_t)g * P.C + (valid ? c : 0)) * L4;

    float lbg[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) lbg[a] = (float)log(P.bg[a]);
    for (int q = 0; q < L4; ++q) {
        Ws[q * NT + tid] = valid ? logf(P.theta_in[c * L4 + q]) - lbg[q & 3] : 0.f;
        if (valid && P.mstep) tot[q] = 0.0;
    }
    double ll = 0.0, zs = 0.0;
    const int i0 = (int)((int64_t)P.t * g / P.G), i1 = (int)((int64_t)P.t * (g + 1) / P.G);
    for (int i = i0; i < i1; ++i) {
        const int64_t base = P.seq_off[i];
        const int ns = P.seq_off[i + 1] - P.seq_off[i] - l + 1;
        if (P.mstep)
            for (int q = 0; q < L4; ++q) { acc[q * NT + tid] = 0.f; cmp[q * NT + tid] = 0.f; }
        float m = -INFINITY, S = 0.f, Sc = 0.f;
        uint64_t win = window64(P.packed, P.nwords, base);
        // next base to shift in is base+32; its word is cached in `nxt`
        int64_t nb = base + 32;
        uint32_t nxt = (nb >> 4) < P.nwords ? __ldg(P.packed + (nb >> 4)) : 0u;
        for (int j = 0; j < ns; ++j) {
            if (j > 0) {
                win = (win >> 2) | ((uint64_t)((nxt >> (2 * (nb & 15))) & 3u) << 62);
                ++nb;
                if ((nb & 15) == 0) nxt = (nb >> 4) < P.nwords ? __ldg(P.packed + (nb >> 4)) : 0u;
            }
            float r = 0.f;
#pragma unroll
            for (int p = 0; p < LMAX; ++p)
                if (p < l) r += Ws[(p * 4 + (int)((win >> (2 * p)) & 3u)) * NT + tid];
            if (r > m) {
                const float sc = expf(m - r);  // 0 on the first l-mer
                S *= sc;
                Sc *= sc;
                if (P.mstep)
                    for (int q = 0; q < L4; ++q) { acc[q * NT + tid] *= sc; cmp[q * NT + tid] *= sc; }
                m = r;
            }
            const float e = expf(r - m);
            kahan_add(S, Sc, e);
            if (P.mstep) {
#pragma unroll
                for (int p = 0; p < LMAX; ++p)
                    if (p < l) {
                        const int q = (p * 4 + (int)((win >> (2 * p)) & 3u)) * NT + tid;
                        float a = acc[q], cc = cmp[q];
                        kahan_add(a, cc, e);
                        acc[q] = a;
                        cmp[q] = cc;
                    }
            }
        }
        const double Sd = (double)S - (double)Sc;
        double w = 1.0;  // posterior probability that the sequence holds a site
        if (P.gamma < 1.0) {
            // ZOOPS: L_i = log[(1 - gamma) + (gamma / ns) sum_j e^r]
            const double lg = log(P.gamma / (double)ns) + (double)m + log(Sd);
            const double Li = log_add_d(log1p(-P.gamma), lg);
            w = exp(lg - Li);
            ll += Li;
        } else {
            ll += (double)m + log(Sd) - log((double)ns);
        }
        zs += w;
        if (P.mstep && valid) {
            const double inv = w / Sd;
            for (int q = 0; q < L4; ++q)
                tot[q] += ((double)acc[q * NT + tid] - (double)cmp[q * NT + tid]) * inv;
        }
    }
    if (valid) {
        P.part_ll[(int64_t)g * P.C + c] = ll;
        P.part_zs[(int64_t)g * P.C + c] = zs;
    }
}

// Sum of the G partial results in group order (fixed, so deterministic), then
// the M-step theta = (counts + pseudocount) / (t + 4 pseudocount).
__global__ void em_reduce_kernel(const double *__restrict__ part_acc,
                                 const double *__restrict__ part_ll,
                                 const double *__restrict__ part_zs, int zoops, int G, int64_t C,
                                 int L4, int t, float beta, int mstep,
                                 float *__restrict__ theta_out, double *__restrict__ ll_out) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (mstep && idx < C * L4) {
        double s = 0.0, sites = (double)t;  // OOPS: one site per sequence
        for (int g = 0; g < G; ++g) s += part_acc[(int64_t)g * C * L4 + idx];
        if (zoops) {
            sites = 0.0;
            for (int g = 0; g < G; ++g) sites += part_zs[(int64_t)g * C + idx / L4];
        }
        theta_out[idx] = (float)((s + (double)beta) / (sites + 4.0 * (double)beta));
    }
    if (idx < C) {
        double s = 0.0;
        for (int g = 0; g < G; ++g) s += part_ll[(int64_t)g * C + idx];
        ll_out[idx] = s;
    }
}

// ---------------------------------------------------------------------------
// Ranking and finalisation (one CTA).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void finalize_body(
    const uint32_t *__restrict__ packed, int64_t nwords, const int32_t *__restrict__ seq_off,
    int t, int l, const double *__restrict__ bg, const float *__restrict__ theta, int stride,
    const double *__restrict__ ll, int64_t C, int64_t *__restrict__ best_out,
    int32_t *__restrict__ sites, uint8_t *__restrict__ consensus, int32_t *__restrict__ score,
    bool with_sites = true) {
    __shared__ double s_v[32];
    __shared__ long long s_i[32];
    __shared__ double W[32 * 4];
    __shared__ long long s_best;
    __shared__ int s_score[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // argmax of the FP64 log-likelihoods; ties to the smaller index
    double bv = -INFINITY;
    long long bi = -1;
    for (int64_t c = tid; c < C; c += blockDim.x) {
        const double v = ll[c];
        if (bi < 0 || v > bv) { bv = v; bi = c; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, o);
        const long long oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
    }
    if (lane == 0) { s_v[warp] = bv; s_i[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
        bv = lane < (int)(blockDim.x / 32) ? s_v[lane] : -INFINITY;
        bi = lane < (int)(blockDim.x / 32) ? s_i[lane] : -1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, bv, o);
            const long long oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
        }
        if (lane == 0) s_best = bi;
    }
    __syncthreads();
    const long long b = s_best;
    if (tid == 0) *best_out = b;
    if (b < 0) {
        if (tid == 0) *score = 0;
        for (int i = tid; i < t; i += blockDim.x) sites[i] = -1;
        for (int p = tid; p < l; p += blockDim.x) consensus[p] = 'N';
        return;
    }
    const float *th = theta + b * (int64_t)stride;
    if (tid < 4 * l) W[tid] = log((double)th[tid]) - log(bg[tid & 3]);
    if (tid < l) {
        int a = 0;
        for (int q = 1; q < 4; ++q) if (th[tid * 4 + q] > th[tid * 4 + a]) a = q;
        consensus[tid] = (uint8_t)("ACTG"[a]);
    }
    __syncthreads();
    if (!with_sites) return;  // sites_kernel and score_kernel follow
    // sites: first start maximising r(i,j), in FP64
    for (int i = warp; i < t; i += blockDim.x / 32) {
        const int64_t base = seq_off[i];
        const int ns = seq_off[i + 1] - seq_off[i] - l + 1;
        double best = -INFINITY;
        int bj = 0x7fffffff;
        for (int j = lane; j < ns; j += 32) {
            const uint64_t win = window64(packed, nwords, base + j);
            double r = 0.0;
            for (int p = 0; p < l; ++p) r += W[p * 4 + (int)((win >> (2 * p)) & 3u)];
            if (r > best) { best = r; bj = j; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_down_sync(0xffffffffu, best, o);
            const int oj = __shfl_down_sync(0xffffffffu, bj, o);
            if (ob > best || (ob == best && oj < bj)) { best = ob; bj = oj; }
        }
        if (lane == 0) sites[i] = ns > 0 ? bj : -1;
    }
    __syncthreads();
    // Score(s, DNA): sum over columns of the largest base count
    int colmax = 0;
    if (tid < l) {
        int cnt[4] = {0, 0, 0, 0};
        for (int i = 0; i < t; ++i) {
            const int a = sites[i];
            if (a >= 0) ++cnt[code_at(packed, nwords, (int64_t)seq_off[i] + a + tid)];
        }
        colmax = max(max(cnt[0], cnt[1]), max(cnt[2], cnt[3]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) colmax += __shfl_down_sync(0xffffffffu, colmax, o);
    if (lane == 0) s_score[warp] = colmax;
    __syncthreads();
    if (tid == 0) {
        int sc = 0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) sc += s_score[w];
        *score = sc;
    }
}

// Sites of the winner, one CTA (one warp) per sequence: the FP64 scoring of
// every l-mer is spread over as many SMs as there are sequences (the FP64
// pipe of this part is narrow).
__global__ void __launch_bounds__(32) sites_kernel(
    const uint32_t *__restrict__ packed, int64_t nwords, const int32_t *__restrict__ seq_off,
    int t, int l, const double *__restrict__ bg, const float *__restrict__ theta,
    const int64_t *__restrict__ best, int32_t *__restrict__ sites) {
    __shared__ double W[32 * 4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long b = *best;
    const int i = blockIdx.x * (blockDim.x / 32) + warp;
    if (b < 0) {
        if (lane == 0 && i < t) sites[i] = -1;
        return;
    }
    const float *th = theta + b * (int64_t)(4 * l);
    for (int q = tid; q < 4 * l; q += blockDim.x) W[q] = log((double)th[q]) - log(bg[q & 3]);
    __syncthreads();
    if (i >= t) return;
    const int64_t base = seq_off[i];
    const int ns = seq_off[i + 1] - seq_off[i] - l + 1;
    double bestv = -INFINITY;
    int bj = 0x7fffffff;
    for (int j = lane; j < ns; j += 32) {
        const uint64_t win = window64(packed, nwords, base + j);
        double r = 0.0;
        for (int p = 0; p < l; ++p) r += W[p * 4 + (int)((win >> (2 * p)) & 3u)];
        if (r > bestv) { bestv = r; bj = j; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, bestv, o);
        const int oj = __shfl_down_sync(0xffffffffu, bj, o);
        if (ob > bestv || (ob == bestv && oj < bj)) { bestv = ob; bj = oj; }
    }
    if (lane == 0) sites[i] = ns > 0 ? bj : -1;
}

// Sites of every candidate (Definition 1's start vector s under each model):
// one CTA per candidate, W = log theta - log bg in FP64 in shared memory, one
// warp per sequence in turn; ties go to the first start, as for the winner.
__global__ void __launch_bounds__(256) cand_sites_kernel(
    const uint32_t *__restrict__ packed, int64_t nwords, const int32_t *__restrict__ seq_off,
    int t, int l, const double *__restrict__ bg, const float *__restrict__ theta,
    int32_t *__restrict__ sites) {
    __shared__ double W[32 * 4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t c = blockIdx.x;
    const float *th = theta + c * (int64_t)(4 * l);
    for (int q = tid; q < 4 * l; q += blockDim.x) W[q] = log((double)th[q]) - log(bg[q & 3]);
    __syncthreads();
    for (int i = warp; i < t; i += blockDim.x / 32) {
        const int64_t base = seq_off[i];
        const int ns = seq_off[i + 1] - seq_off[i] - l + 1;
        double bestv = -INFINITY;
        int bj = 0x7fffffff;
        for (int j = lane; j < ns; j += 32) {
            const uint64_t win = window64(packed, nwords, base + j);
            double r = 0.0;
            for (int p = 0; p < l; ++p) r += W[p * 4 + (int)((win >> (2 * p)) & 3u)];
            if (r > bestv) { bestv = r; bj = j; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_down_sync(0xffffffffu, bestv, o);
            const int oj = __shfl_down_sync(0xffffffffu, bj, o);
            if (ob > bestv || (ob == bestv && oj < bj)) { bestv = ob; bj = oj; }
        }
        if (lane == 0) sites[c * t + i] = ns > 0 ? bj : -1;
    }
}

// Score(s, DNA) of the winner's sites: sum over columns of the largest count.
__global__ void __launch_bounds__(1024) score_kernel(
    const uint32_t *__restrict__ packed, int64_t nwords, const int32_t *__restrict__ seq_off,
    int t, int l, const int32_t *__restrict__ sites, int32_t *__restrict__ score) {
    __shared__ int s_cnt[32 * 4];
    const int tid = threadIdx.x;
    for (int q = tid; q < 4 * l; q += blockDim.x) s_cnt[q] = 0;
    __syncthreads();
    for (int e = tid; e < t * l; e += blockDim.x) {
        const int i = e / l, p = e - i * l;
        const int a = sites[i];
        if (a >= 0) atomicAdd(&s_cnt[p * 4 + code_at(packed, nwords, (int64_t)seq_off[i] + a + p)], 1);
    }
    __syncthreads();
    if (tid == 0) {
        int sc = 0;
        for (int p = 0; p < l; ++p)
            sc += max(max(s_cnt[4 * p], s_cnt[4 * p + 1]), max(s_cnt[4 * p + 2], s_cnt[4 * p + 3]));
        *score = sc;
    }
}

__global__ void __launch_bounds__(1024) finalize_kernel(
    const uint32_t *__restrict__ packed, int64_t nwords, const int32_t *__restrict__ seq_off,
    int t, int l, const double *__restrict__ bg, const float *__restrict__ theta,
    const double *__restrict__ ll, int64_t C, int64_t *__restrict__ best_out,
    int32_t *__restrict__ sites, uint8_t *__restrict__ consensus, int32_t *__restrict__ score) {
    finalize_body(packed, nwords, seq_off, t, l, bg, theta, 4 * l, ll, C, best_out, sites,
                  consensus, score, false);
}

// One CTA per instance of a batch.
__global__ void __launch_bounds__(1024) finalize_batch_kernel(
    const uint32_t *__restrict__ packed, int64_t nwords, const BatchInst *__restrict__ inst,
    const float *__restrict__ theta, int stride, const double *__restrict__ ll,
    int64_t *__restrict__ best_out, int32_t *__restrict__ sites, uint8_t *__restrict__ consensus,
    int32_t *__restrict__ score) {
    const BatchInst in = inst[blockIdx.x];
    finalize_body(packed, nwords, in.seq_off, in.t, in.l, in.bg, theta + in.cand_begin * stride,
                  stride, ll + in.cand_begin, in.C, best_out + blockIdx.x, sites + in.sites_off,
                  consensus + in.cons_off, score + blockIdx.x);
}

// theta^0 for the candidates of all instances of a batch (models at `stride`).
__global__ void theta0_batch_kernel(const uint32_t *__restrict__ packed, int64_t nwords,
                                    const BatchInst *__restrict__ inst, int n_inst,
                                    const int64_t *__restrict__ cand_off,
                                    const int32_t *__restrict__ members, int64_t C, float beta,
                                    int stride, float *__restrict__ theta0) {
    extern __shared__ float cnt[];  // [stride][blockDim]
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t c = blockIdx.x * (int64_t)nt + tid;
    for (int q = 0; q < stride; ++q) cnt[q * nt + tid] = 0.f;
    if (c >= C) return;
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (inst[mid].cand_begin <= c) lo = mid; else hi = mid - 1;
    }
    const BatchInst in = inst[lo];
    const int l = in.l;
    const int64_t e0 = cand_off[c], e1 = cand_off[c + 1];
    for (int64_t e = e0; e < e1; ++e) {
        const int g = members[e];
        int a = 0, b = in.t - 1;  // last sequence with lmer_off <= g
        while (a < b) {
            const int mid = (a + b + 1) >> 1;
            if (__ldg(in.lmer_off + mid) <= g) a = mid; else b = mid - 1;
        }
        const int64_t b0 = (int64_t)__ldg(in.seq_off + a) + (g - __ldg(in.lmer_off + a));
        const uint64_t win = window64(packed, nwords, b0);
        for (int p = 0; p < l; ++p) cnt[(p * 4 + (int)((win >> (2 * p)) & 3u)) * nt + tid] += 1.f;
    }
    const float den = (float)(e1 - e0) + 4.f * beta;
    for (int q = 0; q < stride; ++q)
        theta0[c * stride + q] = q < 4 * l ? (cnt[q * nt + tid] + beta) / den : 0.f;
}

template <int LMAX>
int launch_em_fp32_iter(const EmParams &P, cudaStream_t st) {
    const size_t smem = (size_t)3 * 4 * P.l * kEmThreads * sizeof(float);
    PROJ_CUDA_TRY(cudaFuncSetAttribute(em_fp32_kernel<LMAX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((unsigned)((P.C + kEmThreads - 1) / kEmThreads), (unsigned)P.G);
    {
        TraceSpan ts_("em_fp32", st);
        em_fp32_kernel<LMAX><<<grid, kEmThreads, smem, st>>>(P);
    }
    PROJ_LAUNCH_CHECK("em_fp32_kernel");
    return PROJ_OK;
}

}  // namespace

// Up to this many candidates theta0 takes one warp per candidate (searches that
// keep a few large buckets); beyond it one thread per candidate, whose buckets
// hold a few l-mers each.
constexpr int64_t kTheta0WarpMaxC = 65536;

int launch_theta0(const uint32_t *packed, const Layout &L, const int64_t *cand_off,
                  const int32_t *members, int64_t C, float beta, float *theta0, cudaStream_t st) {
    if (C == 0) return PROJ_OK;
    if (C <= kTheta0WarpMaxC) {  // few candidates: one warp each
        {
            TraceSpan ts_("theta0", st);
            theta0_warp_kernel<<<(unsigned)((C + 7) / 8), 256, 0, st>>>(
                packed, L.nwords, L.seq_off_dev(), L.lmer_off_dev(), L.t, L.l, cand_off, members, C,
                beta, theta0);
        }
        PROJ_LAUNCH_CHECK("theta0_warp_kernel");
        return PROJ_OK;
    }
    const int nt = 128;
    const size_t smem = (size_t)4 * L.l * nt * sizeof(float);
    PROJ_CUDA_TRY(cudaFuncSetAttribute(theta0_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    {
        TraceSpan ts_("theta0", st);
        theta0_kernel<<<(unsigned)((C + nt - 1) / nt), nt, smem, st>>>(
            packed, L.nwords, L.seq_off_dev(), L.lmer_off_dev(), L.t, L.l, cand_off, members, C, beta,
            theta0);
    }
    PROJ_LAUNCH_CHECK("theta0_kernel");
    return PROJ_OK;
}

int run_em(const uint32_t *packed, const Layout &L, const double *bg, const float *theta0,
           int64_t C, int iters, float beta, int precision, float *theta_out, double *ll,
           cudaStream_t st, double gamma, int *err_dev) {
    PROJ_REQUIRE(iters >= 0 && iters <= 1000, "em_iters out of range: %d", iters);
    PROJ_REQUIRE(beta > 0.f, "pseudocount must be > 0");
    PROJ_REQUIRE(precision == PROJ_EM_FP32 || precision == PROJ_EM_BF16_SPLIT,
                 "unknown precision %d", precision);
    if (C == 0) return PROJ_OK;
    PROJ_REQUIRE(gamma > 0.0 && gamma <= 1.0, "site probability must be in (0, 1]");
    if (precision == PROJ_EM_BF16_SPLIT)
        return run_em_tc(packed, L, bg, theta0, C, iters, beta, theta_out, ll, st, gamma, err_dev);

    const int L4 = 4 * L.l;
    // enough (candidate-tile, sequence-group) units to fill every SM a few times
    const int64_t tiles = (C + kEmThreads - 1) / kEmThreads;
    const int64_t want = (int64_t)sm_count() * 8;
    const int G = (int)std::min<int64_t>(L.t, std::max<int64_t>(1, (want + tiles - 1) / tiles));
    DevBuf part;
    PROJ_TRY(part.alloc((size_t)G * C * (L4 + 2) * sizeof(double), st));
    DevBuf tmp;  // model of the current iteration (theta_out may alias theta0)
    PROJ_TRY(tmp.alloc((size_t)C * L4 * sizeof(float), st));
    PROJ_CUDA_TRY(cudaMemcpyAsync(tmp.as<float>(), theta0, (size_t)C * L4 * sizeof(float),
                                  cudaMemcpyDeviceToDevice, st));

    EmParams P{};
    P.packed = packed;
    P.nwords = L.nwords;
    P.seq_off = L.seq_off_dev();
    P.t = L.t;
    P.l = L.l;
    P.G = G;
    P.bg = bg;
    P.C = C;
    P.part_ll = part.as<double>();
    P.part_zs = part.as<double>() + (size_t)G * C;
    P.part_acc = part.as<double>() + (size_t)2 * G * C;
    P.gamma = gamma;
    P.theta_in = tmp.as<float>();
    for (int it = 0; it <= iters; ++it) {
        P.mstep = it < iters;
        int rc;
        if (L.l <= 8) rc = launch_em_fp32_iter<8>(P, st);
        else if (L.l <= 16) rc = launch_em_fp32_iter<16>(P, st);
        else if (L.l <= 24) rc = launch_em_fp32_iter<24>(P, st);
        else rc = launch_em_fp32_iter<32>(P, st);
        if (rc != PROJ_OK) return rc;
        const int64_t n = P.mstep ? C * L4 : C;
        {
            TraceSpan ts_("em_reduce", st);
            em_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                P.part_acc, P.part_ll, P.part_zs, gamma < 1.0 ? 1 : 0, G, C, L4, L.t, beta,
                P.mstep, tmp.as<float>(), ll);
        }
        PROJ_LAUNCH_CHECK("em_reduce_kernel");
    }
    PROJ_CUDA_TRY(cudaMemcpyAsync(theta_out, tmp.as<float>(), (size_t)C * L4 * sizeof(float),
                                  cudaMemcpyDeviceToDevice, st));
    return PROJ_OK;
}

int launch_theta0_batch(const uint32_t *packed, int64_t nwords, const BatchInst *inst, int n_inst,
                        const int64_t *cand_off, const int32_t *members, int64_t C, float beta,
                        int stride, float *theta0, cudaStream_t st) {
    if (C == 0) return PROJ_OK;
    const int nt = 128;
    const size_t smem = (size_t)stride * nt * sizeof(float);
    PROJ_CUDA_TRY(cudaFuncSetAttribute(theta0_batch_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
        TraceSpan ts_("theta0", st);
        theta0_batch_kernel<<<(unsigned)((C + nt - 1) / nt), nt, smem, st>>>(
            packed, nwords, inst, n_inst, cand_off, members, C, beta, stride, theta0);
    }
    PROJ_LAUNCH_CHECK("theta0_batch_kernel");
    return PROJ_OK;
}

int launch_finalize_batch(const uint32_t *packed, int64_t nwords, const BatchInst *inst,
                          int n_inst, const float *theta, int stride, const double *ll,
                          int64_t *best, int32_t *sites, uint8_t *consensus, int32_t *score,
                          cudaStream_t st) {
    {
        TraceSpan ts_("finalize", st);
        finalize_batch_kernel<<<n_inst, 1024, 0, st>>>(packed, nwords, inst, theta, stride, ll, best,
                                                       sites, consensus, score);
    }
    PROJ_LAUNCH_CHECK("finalize_batch_kernel");
    return PROJ_OK;
}

int launch_finalize(const uint32_t *packed, const Layout &L, const double *bg,
                    const float *theta, const double *ll, int64_t C, int64_t *best,
                    int32_t *sites, uint8_t *consensus, int32_t *score, cudaStream_t st) {
    PROJ_REQUIRE(L.l <= 32, "l above 32 is not supported");
    {
        TraceSpan ts_("finalize", st);
        finalize_kernel<<<1, 1024, 0, st>>>(packed, L.nwords, L.seq_off_dev(), L.t, L.l, bg, theta, ll,
                                            C, best, sites, consensus, score);
    }
    PROJ_LAUNCH_CHECK("finalize_kernel");
    {
        TraceSpan ts_("finalize", st);
        sites_kernel<<<(unsigned)L.t, 32, 0, st>>>(packed, L.nwords, L.seq_off_dev(), L.t, L.l, bg,
                                                    theta, best, sites);
    }
    PROJ_LAUNCH_CHECK("sites_kernel");
    {
        TraceSpan ts_("finalize", st);
        score_kernel<<<1, 1024, 0, st>>>(packed, L.nwords, L.seq_off_dev(), L.t, L.l, sites, score);
    }
    PROJ_LAUNCH_CHECK("score_kernel");
    return PROJ_OK;
}

int launch_cand_sites(const uint32_t *packed, const Layout &L, const double *bg,
                      const float *theta, int64_t C, int32_t *sites, cudaStream_t st) {
    PROJ_REQUIRE(L.l <= 32, "l above 32 is not supported");
    PROJ_REQUIRE(C < ((int64_t)1 << 31), "too many candidates");
    if (C == 0) return PROJ_OK;
    {
        TraceSpan ts_("cand_sites", st);
        cand_sites_kernel<<<(unsigned)C, 256, 0, st>>>(packed, L.nwords, L.seq_off_dev(), L.t, L.l,
                                                       bg, theta, sites);
    }
    PROJ_LAUNCH_CHECK("cand_sites_kernel");
    return PROJ_OK;
}

}  // namespace proj
