// The motif search over the 20-letter protein alphabet (Section 2: |Sigma| = 20
// for proteins; letters ACDEFGHIKLMNPQRSTVWY with codes 0..19).  Residues are
// kept one per byte; keys are base 20, so 20^k buckets leave no room for a
// histogram and the enriched buckets come from a per-trial sort of (key,
// l-mer) pairs in shared memory, or the all-pairs comparison beyond 16,384
// l-mers (csrc/allpairs.cu, k <= 6).  theta^0 and OOPS EM (Section 5.1) score in
// FP32 over 20l weights per model; ranking and sites are FP64, as for DNA.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace proj {
namespace {

constexpr int kAA = 20;

// ASCII -> codes 0..19 (either case); the smallest index of another character
// goes to *bad (initialised to a large value by the host).
__global__ void aa_pack_kernel(const uint8_t *__restrict__ ascii, int64_t n,
                               uint8_t *__restrict__ codes, unsigned long long *__restrict__ bad) {
    // code of each upper-case letter, 255 = not an amino-acid letter
    constexpr uint8_t X = 255;
    const uint8_t table[26] = {0, X, 1, 2, 3, 4, 5, 6, 7, X, 8, 9, 10, 11, X, 12, 13, 14, 15, 16,
                               X, 17, 18, X, 19, X};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int ch = ascii[i];
        if (ch >= 'a' && ch <= 'z') ch -= 32;
        const uint8_t c = (ch >= 'A' && ch <= 'Z') ? table[ch - 'A'] : X;
        if (c == X) atomicMin(bad, (unsigned long long)i);
        codes[i] = c == X ? 0 : c;
    }
}

// 0-order residue frequencies (an absent residue counts once, as for DNA).
__global__ void aa_background_kernel(const uint8_t *__restrict__ codes, int64_t n,
                                     double *__restrict__ bg) {
    __shared__ unsigned int cnt[kAA];  // inputs hold < 2^31 residues
    if (threadIdx.x < kAA) cnt[threadIdx.x] = 0u;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&cnt[codes[i]], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int a = 0; a < kAA; ++a) { if (cnt[a] == 0u) cnt[a] = 1u; tot += cnt[a]; }
        for (int a = 0; a < kAA; ++a) bg[a] = (double)cnt[a] / (double)tot;
    }
}

// theta^0 = (letter counts of the bucket's l-mers + beta) / (cnt + 20 beta),
// one warp per candidate (integer counts: the order of the atomics is immaterial).
__global__ void aa_theta0_kernel(const uint8_t *__restrict__ codes,
                                 const int32_t *__restrict__ seq_off,
                                 const int32_t *__restrict__ lmer_off, int t, int l,
                                 const int64_t *__restrict__ cand_off,
                                 const int32_t *__restrict__ members, int64_t C, float beta,
                                 float *__restrict__ theta0) {
    __shared__ int cnt[8][kAA * 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = blockIdx.x * 8 + warp;
    if (c >= C) return;
    int *h = cnt[warp];
    for (int q = lane; q < kAA * l; q += 32) h[q] = 0;
    __syncwarp();
    const int64_t e0 = cand_off[c], e1 = cand_off[c + 1];
    for (int64_t e = e0 + lane; e < e1; e += 32) {
        const int g = members[e];
        int lo = 0, hi = t - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(lmer_off + mid) <= g) lo = mid; else hi = mid - 1;
        }
        const uint8_t *lmer = codes + __ldg(seq_off + lo) + (g - __ldg(lmer_off + lo));
        for (int p = 0; p < l; ++p) atomicAdd(&h[p * kAA + lmer[p]], 1);
    }
    __syncwarp();
    const float den = (float)(e1 - e0) + (float)kAA * beta;
    for (int q = lane; q < kAA * l; q += 32) theta0[c * kAA * l + q] = ((float)h[q] + beta) / den;
}

// One OOPS EM iteration (E-step + optional M-step) for one candidate per CTA.
// Warps take sequences in turn, lanes take l-mers: pass A gives every lane a
// running (max, sum) of e^r in FP32 (r = sum_p W[p][x], W = log theta - log
// bg), merged across lanes into L_i = log sum_j e^{r(i,j)}; pass B
// recomputes r and adds z = e^{r - L_i} to the counts of the l letters of its
// l-mer.  Counts are fixed point in units of 2^-31: a warp sums its current
// sequence with 32-bit integer atomics (a sequence's z sum to 1, so every
// count stays below 2^32) and adds the sequence's counts to the CTA's 64-bit
// totals.  Integer sums do not depend on the order of the additions, and the
// per-warp log-likelihoods are summed in warp order, so results are
// deterministic.  The M-step writes theta = (counts + beta) / (t + 20 beta)
// (Section 5.1) directly.  Transcendentals and divisions are FP32 (the FP64
// pipe of this part runs 2 lanes per clock per SM); the per-sequence terms
// are summed in FP64.
constexpr int kAaEmThreads = 256;
constexpr int kAaEmWarps = kAaEmThreads / 32;
constexpr float kFix = 2147483648.f;  // 2^31

__global__ void __launch_bounds__(kAaEmThreads) aa_em_kernel(
    const uint8_t *__restrict__ codes, const int32_t *__restrict__ seq_off, int t, int l,
    const double *bg, const float *theta_in, float beta, int mstep, float *theta_out,
    double *__restrict__ ll_out) {
    __shared__ float W[kAA * 32];
    __shared__ unsigned long long acc[kAA * 32];
    __shared__ unsigned int seq_acc[kAaEmWarps][kAA * 32];
    __shared__ double s_ll[kAaEmWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L20 = kAA * l;
    const int64_t c = blockIdx.x;
    unsigned int *a32 = seq_acc[warp];
    for (int q = tid; q < L20; q += kAaEmThreads) {
        W[q] = logf(theta_in[c * L20 + q]) - logf((float)bg[q % kAA]);
        acc[q] = 0ull;
    }
    for (int q = lane; q < L20; q += 32) a32[q] = 0u;
    __syncthreads();
    double ll = 0.0;
    for (int i = warp; i < t; i += kAaEmWarps) {
        const uint8_t *seq = codes + seq_off[i];
        const int ns = seq_off[i + 1] - seq_off[i] - l + 1;
        float m = -INFINITY, S = 0.f;
        for (int j = lane; j < ns; j += 32) {
            float r = 0.f;
            for (int p = 0; p < l; ++p) r += W[p * kAA + seq[j + p]];
            if (r > m) {
                S = S * expf(m - r) + 1.f;
                m = r;
            } else {
                S += expf(r - m);
            }
        }
        float M = m;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) M = fmaxf(M, __shfl_xor_sync(0xffffffffu, M, o));
        float Sf = S > 0.f ? S * expf(m - M) : 0.f;  // lane sums relative to the warp maximum
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) Sf += __shfl_xor_sync(0xffffffffu, Sf, o);
        ll += (double)(M + logf(Sf) - logf((float)ns));
        if (mstep) {
            const float scale = kFix / Sf;
            for (int j = lane; j < ns; j += 32) {
                float r = 0.f;
                for (int p = 0; p < l; ++p) r += W[p * kAA + seq[j + p]];
                const unsigned int z = __float2uint_rn(expf(r - M) * scale);
                for (int p = 0; p < l; ++p) atomicAdd(&a32[p * kAA + seq[j + p]], z);
            }
            __syncwarp();
            for (int q = lane; q < L20; q += 32) {
                const unsigned int v = a32[q];
                if (v) {
                    atomicAdd(&acc[q], (unsigned long long)v);
                    a32[q] = 0u;
                }
            }
            __syncwarp();
        }
    }
    if (lane == 0) s_ll[warp] = ll;
    __syncthreads();
    if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < kAaEmWarps; ++w) tot += s_ll[w];
        ll_out[c] = tot;
    }
    if (mstep) {
        const float inv = 1.f / ((float)t + (float)kAA * beta);
        for (int q = tid; q < L20; q += kAaEmThreads)
            theta_out[c * L20 + q] = ((float)acc[q] * (1.f / kFix) + beta) * inv;
    }
}

// FP64 argmax of the log-likelihoods (ties to the smaller index) and the
// winner's consensus (per column the letter of largest weight, ties to the
// lowest code).
__global__ void __launch_bounds__(1024) aa_rank_kernel(const double *__restrict__ ll, int64_t C,
                                                       const float *__restrict__ theta, int l,
                                                       int64_t *__restrict__ best,
                                                       uint8_t *__restrict__ consensus) {
    __shared__ double s_v[32];
    __shared__ long long s_i[32];
    __shared__ long long s_best;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
        bv = s_v[lane];
        bi = s_i[lane];
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
    if (tid == 0) *best = b;
    if (tid < l) {
        const char letters[] = "ACDEFGHIKLMNPQRSTVWY";
        if (b < 0) {
            consensus[tid] = 'X';
        } else {
            const float *th = theta + b * (int64_t)kAA * l + tid * kAA;
            int a = 0;
            for (int q = 1; q < kAA; ++q) if (th[q] > th[a]) a = q;
            consensus[tid] = (uint8_t)letters[a];
        }
    }
}

// Sites of the winner: per sequence the first start of highest FP64 score (one
// CTA of one warp per sequence, spreading the FP64 work over the SMs).
__global__ void __launch_bounds__(256) aa_sites_kernel(const uint8_t *__restrict__ codes,
                                                       const int32_t *__restrict__ seq_off, int t,
                                                       int l, const double *__restrict__ bg,
                                                       const float *__restrict__ theta,
                                                       const int64_t *__restrict__ best,
                                                       int32_t *__restrict__ sites) {
    __shared__ double W[kAA * 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long b = *best;
    const int i = blockIdx.x * (blockDim.x / 32) + warp;
    if (b < 0) {
        if (lane == 0 && i < t) sites[i] = -1;
        return;
    }
    for (int q = tid; q < kAA * l; q += blockDim.x)
        W[q] = log((double)theta[b * (int64_t)kAA * l + q]) - log(bg[q % kAA]);
    __syncthreads();
    if (i >= t) return;
    const uint8_t *seq = codes + seq_off[i];
    const int ns = seq_off[i + 1] - seq_off[i] - l + 1;
    double bestv = -INFINITY;
    int bj = 0x7fffffff;
    for (int j = lane; j < ns; j += 32) {
        double r = 0.0;
        for (int p = 0; p < l; ++p) r += W[p * kAA + seq[j + p]];
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

__global__ void __launch_bounds__(1024) aa_score_kernel(const uint8_t *__restrict__ codes,
                                                        const int32_t *__restrict__ seq_off, int t,
                                                        int l, const int32_t *__restrict__ sites,
                                                        int32_t *__restrict__ score) {
    __shared__ int cnt[kAA * 32];
    for (int q = threadIdx.x; q < kAA * l; q += blockDim.x) cnt[q] = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < t * l; e += blockDim.x) {
        const int i = e / l, p = e - i * l;
        if (sites[i] >= 0) atomicAdd(&cnt[p * kAA + codes[seq_off[i] + sites[i] + p]], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int sc = 0;
        for (int p = 0; p < l; ++p) {
            int mx = 0;
            for (int a = 0; a < kAA; ++a) mx = max(mx, cnt[p * kAA + a]);
            sc += mx;
        }
        *score = sc;
    }
}

int protein_impl(const uint8_t *ascii, const int64_t *seq_off, int t, int l, int k, int s, int m,
                 uint64_t seed, int em_iters, float beta, projection_result *out,
                 cudaStream_t st) {
    PROJ_REQUIRE(ascii != nullptr, "ascii must not be NULL");
    PROJ_REQUIRE(k >= 1 && k <= 6 && k <= l, "need 1 <= k <= min(l, 6) for 20^k keys");
    PROJ_REQUIRE(s >= 1 && m >= 1 && m <= 65535, "need s >= 1 and 1 <= m <= 65535");
    PROJ_REQUIRE(em_iters >= 0 && em_iters <= 1000 && beta > 0.f,
                 "need 0 <= em_iters <= 1000 and pseudocount > 0");
    Layout L;
    PROJ_TRY(make_layout(seq_off, t, l, st, L));
    out->t = t; out->l = l; out->k = k; out->s = s; out->m = m;
    const int64_t total = L.total;

    DevBuf in;  // ascii | codes | bad | bg[20] | totals[2] | best | score | sites[t] | consensus
    const size_t off_codes = (size_t)((total + 15) & ~(int64_t)15);
    const size_t off_tail = off_codes + (size_t)((total + 15) & ~(int64_t)15);
    PROJ_TRY(in.alloc(off_tail + 8 + kAA * 8 + 16 + 8 + 8 + (size_t)t * 4 + (size_t)l + 64, st));
    uint8_t *ascii_dev = in.as<uint8_t>();
    uint8_t *codes = ascii_dev + off_codes;
    unsigned long long *bad = reinterpret_cast<unsigned long long *>(ascii_dev + off_tail);
    double *bg = reinterpret_cast<double *>(bad + 1);
    int64_t *totals = reinterpret_cast<int64_t *>(bg + kAA);
    int64_t *best = totals + 2;
    int32_t *score = reinterpret_cast<int32_t *>(best + 1);
    int32_t *sites = score + 2;
    uint8_t *cons = reinterpret_cast<uint8_t *>(sites + t);
    PROJ_CUDA_TRY(cudaMemcpyAsync(ascii_dev, ascii, (size_t)total, cudaMemcpyHostToDevice, st));
    PROJ_CUDA_TRY(cudaMemsetAsync(bad, 0xFF, 8, st));
    {
        TraceSpan ts_("pack", st);
        aa_pack_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, st>>>(
            ascii_dev, total, codes, bad);
    }
    PROJ_LAUNCH_CHECK("aa_pack_kernel");
    unsigned long long bad_h = 0;
    PROJ_CUDA_TRY(cudaMemcpyAsync(&bad_h, bad, 8, cudaMemcpyDeviceToHost, st));
    PROJ_CUDA_TRY(cudaStreamSynchronize(st));
    if (bad_h != ~0ull) {
        set_error("character %d at index %llu is not an amino-acid letter", (int)ascii[bad_h], bad_h);
        return PROJ_EBADCHAR;
    }
    {
        TraceSpan ts_("background", st);
        aa_background_kernel<<<1, 1024, 0, st>>>(codes, total, bg);
    }
    PROJ_LAUNCH_CHECK("aa_background_kernel");

    // enriched buckets in one pass: a trial has at most x / s candidates and
    // its members are distinct l-mers
    const int64_t cap_c = m * std::max<int64_t>(1, L.x / s), cap_m = m * L.x;
    DevBuf cand;
    PROJ_TRY(cand.alloc((size_t)cap_c * 12 + (size_t)(cap_c + 1) * 8 + (size_t)cap_m * 4 + 64, st));
    int64_t *cand_off = cand.as<int64_t>();
    int32_t *cand_trial = reinterpret_cast<int32_t *>(cand_off + cap_c + 1);
    uint32_t *cand_key = reinterpret_cast<uint32_t *>(cand_trial + cap_c);
    int32_t *cand_cnt = reinterpret_cast<int32_t *>(cand_key + cap_c);
    int32_t *members = cand_cnt + cap_c;
    PROJ_TRY(run_allpairs(nullptr, codes, kAA, L, k, s, seed, 0, m, cap_c, cap_m, cand_trial,
                          cand_key, cand_cnt, cand_off, members, totals, st));
    int64_t tot_h[2];
    PROJ_CUDA_TRY(cudaMemcpyAsync(tot_h, totals, sizeof tot_h, cudaMemcpyDeviceToHost, st));
    PROJ_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t C = tot_h[0], M = tot_h[1];
    PROJ_REQUIRE(C <= cap_c && M <= cap_m, "enriched-bucket lists exceed their bounds");
    out->n_candidates = C;
    out->n_members = M;
    out->n_refined = C;

    const int L20 = kAA * l;
    DevBuf model;
    PROJ_TRY(model.alloc((size_t)std::max<int64_t>(1, C) * (L20 * 4 + 8) + 16, st));
    double *ll = model.as<double>();
    float *theta = reinterpret_cast<float *>(ll + std::max<int64_t>(1, C));
    if (C > 0) {
        {
            TraceSpan ts_("theta0", st);
            aa_theta0_kernel<<<(unsigned)((C + 7) / 8), 256, 0, st>>>(
                codes, L.seq_off_dev(), L.lmer_off_dev(), t, l, cand_off, members, C, beta, theta);
        }
        PROJ_LAUNCH_CHECK("aa_theta0_kernel");
        // in place: a CTA reads its own candidate's model before it writes it
        for (int it = 0; it <= em_iters; ++it) {
            const int mstep = it < em_iters;
            {
                TraceSpan ts_("em_fp32", st);
                aa_em_kernel<<<(unsigned)C, kAaEmThreads, 0, st>>>(codes, L.seq_off_dev(), t, l, bg,
                                                                 theta, beta, mstep, theta, ll);
            }
            PROJ_LAUNCH_CHECK("aa_em_kernel");
        }
    }
    {
        TraceSpan ts_("finalize", st);
        aa_rank_kernel<<<1, 1024, 0, st>>>(ll, C, theta, l, best, cons);
    }
    PROJ_LAUNCH_CHECK("aa_rank_kernel");
    {
        TraceSpan ts_("finalize", st);
        aa_sites_kernel<<<(unsigned)t, 32, 0, st>>>(codes, L.seq_off_dev(), t, l, bg,
                                                                theta, best, sites);
    }
    PROJ_LAUNCH_CHECK("aa_sites_kernel");
    {
        TraceSpan ts_("finalize", st);
        aa_score_kernel<<<1, 1024, 0, st>>>(codes, L.seq_off_dev(), t, l, sites, score);
    }
    PROJ_LAUNCH_CHECK("aa_score_kernel");

    int64_t b = -1;
    PROJ_CUDA_TRY(cudaMemcpyAsync(&b, best, 8, cudaMemcpyDeviceToHost, st));
    PROJ_CUDA_TRY(cudaStreamSynchronize(st));
    out->win_index = b;
    out->pwm = (float *)calloc((size_t)L20, sizeof(float));
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
        PROJ_CUDA_TRY(cudaMemcpyAsync(out->pwm, theta + b * L20, (size_t)L20 * 4,
                                      cudaMemcpyDeviceToHost, st));
        PROJ_CUDA_TRY(cudaMemcpyAsync(&out->loglik, ll + b, 8, cudaMemcpyDeviceToHost, st));
        PROJ_CUDA_TRY(cudaMemcpyAsync(&out->win_trial, cand_trial + b, 4, cudaMemcpyDeviceToHost, st));
        PROJ_CUDA_TRY(cudaMemcpyAsync(&out->win_key, cand_key + b, 4, cudaMemcpyDeviceToHost, st));
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

}  // namespace
}  // namespace proj

using namespace proj;

extern "C" int projection_find_protein(const uint8_t *ascii, const int64_t *seq_off, int t, int l,
                                       int k, int s, int m, uint64_t seed, int em_iters,
                                       float pseudocount, projection_result *out, void *stream) {
    clear_error();
    if (!out) { set_error("out must not be NULL"); return PROJ_EINVAL; }
    memset(out, 0, sizeof *out);
    out->win_index = -1;
    out->win_trial = -1;
    const int rc = protein_impl(ascii, seq_off, t, l, k, s, m, seed, em_iters, pseudocount, out,
                                (cudaStream_t)stream);
    out->status = rc;
    return rc;
}
