// Low-memory enrichment by all-pairs comparison (PROJECTION2 of Section 5.2 /
// the per-thread k-mer comparison of Section 6's CUDA-PROJECTION): no 4^k
// table; per trial O(x) memory and O(x^2) comparisons.  Same output as
// trial_hash: the enriched buckets of each trial in key order with their
// member l-mers ascending, bit for bit.
//
//   ap_keys_kernel     keys of every l-mer of every trial (Algorithm 2 step 2b)
//   ap_compare_kernel  per l-mer over all l-mers of its trial: bucket size,
//                      rank among equal keys, first l-mer of the bucket
//   ap_trial_kernel    per trial: enriched buckets (first l-mers with size >= s)
//                      compacted, sorted by key, member offsets
//   ap_scan_kernel     offsets of every trial's candidates and members
//   ap_write_kernel    candidate table; ap_members_kernel member lists
// The protein search (20-letter keys) takes a sort path instead when a trial's
// l-mers fit one CTA's shared memory (x <= 16384): se_sort_kernel sorts the
// trial's (key, l-mer) pairs (bitonic, O(x log^2 x)) and counts its enriched
// runs, se_write_kernel writes the same candidate table and member lists.
#include <algorithm>

#include "common.cuh"

namespace proj {
namespace {

constexpr int kApThreads = 256;
constexpr int kApTrialThreads = 1024;
constexpr int kApMaxBuckets = 4096;  // enriched buckets per trial this mode supports

__device__ __forceinline__ uint32_t ap_key(uint64_t win, const int *pos, int k) {
    uint32_t key = 0u;
#pragma unroll
    for (int q = 0; q < 16; ++q)
        if (q < k) key = (key << 2) | (uint32_t)((win >> (2 * pos[q])) & 3u);
    return key;
}

__global__ void __launch_bounds__(kApThreads) ap_keys_kernel(
    const uint32_t *__restrict__ packed, int64_t nwords, const int32_t *__restrict__ seq_off,
    const int32_t *__restrict__ lmer_off, int t, int l, int k, int x, uint64_t seed,
    int64_t trial_begin, uint32_t *__restrict__ keys) {
    __shared__ int s_pos[16];
    const int trial_local = blockIdx.y;
    if (threadIdx.x == 0) draw_positions(seed, (uint64_t)(trial_begin + trial_local), l, k, s_pos);
    __syncthreads();
    int pos[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) pos[q] = q < k ? s_pos[q] : 0;
    const int g = blockIdx.x * kApThreads + threadIdx.x;
    if (g >= x) return;
    int lo = 0, hi = t - 1;  // sequence of l-mer g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(lmer_off + mid) <= g) lo = mid; else hi = mid - 1;
    }
    const int64_t b0 = (int64_t)__ldg(seq_off + lo) + (g - __ldg(lmer_off + lo));
    keys[(int64_t)trial_local * x + g] = ap_key(window64(packed, nwords, b0), pos, k);
}

// Keys over the 20-letter protein alphabet: byte codes 0..19, base 20, the
// first projected position most significant.
__global__ void __launch_bounds__(kApThreads) ap_keys_aa_kernel(
    const uint8_t *__restrict__ codes, const int32_t *__restrict__ seq_off,
    const int32_t *__restrict__ lmer_off, int t, int l, int k, int x, uint64_t seed,
    int64_t trial_begin, uint32_t *__restrict__ keys) {
    __shared__ int s_pos[16];
    const int trial_local = blockIdx.y;
    if (threadIdx.x == 0) draw_positions(seed, (uint64_t)(trial_begin + trial_local), l, k, s_pos);
    __syncthreads();
    const int g = blockIdx.x * kApThreads + threadIdx.x;
    if (g >= x) return;
    int lo = 0, hi = t - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(lmer_off + mid) <= g) lo = mid; else hi = mid - 1;
    }
    const uint8_t *lmer = codes + __ldg(seq_off + lo) + (g - __ldg(lmer_off + lo));
    uint32_t key = 0u;
    for (int q = 0; q < k; ++q) key = key * 20u + (uint32_t)lmer[s_pos[q]];
    keys[(int64_t)trial_local * x + g] = key;
}

// The comparison of l-mer g's projected k-mer with those of all x l-mers of
// its trial, taken through shared memory one tile at a time.
__global__ void __launch_bounds__(kApThreads) ap_compare_kernel(const uint32_t *__restrict__ keys,
                                                                int x, int32_t *__restrict__ cnt,
                                                                int32_t *__restrict__ rank,
                                                                int32_t *__restrict__ lead) {
    __shared__ uint32_t tile[kApThreads];
    const int64_t base = (int64_t)blockIdx.y * x;
    const int g = blockIdx.x * kApThreads + threadIdx.x;
    const uint32_t kg = g < x ? keys[base + g] : 0u;
    int c = 0, r = 0, first = -1;
    for (int h0 = 0; h0 < x; h0 += kApThreads) {
        __syncthreads();
        if (h0 + (int)threadIdx.x < x) tile[threadIdx.x] = keys[base + h0 + threadIdx.x];
        __syncthreads();
        const int n = min(kApThreads, x - h0);
        for (int q = 0; q < n; ++q) {
            if (tile[q] == kg) {
                ++c;
                if (h0 + q < g) ++r;
                if (first < 0) first = h0 + q;
            }
        }
    }
    if (g < x) {
        cnt[base + g] = c;
        rank[base + g] = r;
        lead[base + g] = first;
    }
}

// One CTA per trial: the enriched buckets' first l-mers in l-mer order
// (ballot scan), sorted by key (bitonic sort in shared memory), and the
// bucket-order prefix of their sizes.  Writes list[trial][i] = (key, g) and
// lsize/loff, nb[trial], nm[trial]; flags err when a trial has more than
// kApMaxBuckets enriched buckets.
__global__ void __launch_bounds__(kApTrialThreads) ap_trial_kernel(
    const uint32_t *__restrict__ keys, const int32_t *__restrict__ cnt,
    const int32_t *__restrict__ rank, int x, int s, uint2 *__restrict__ list,
    int32_t *__restrict__ lsize, int32_t *__restrict__ loff, int32_t *__restrict__ nb,
    int32_t *__restrict__ nm, int *__restrict__ err) {
    __shared__ uint32_t s_key[kApMaxBuckets];
    __shared__ int32_t s_g[kApMaxBuckets];
    __shared__ int s_w[33];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * x;
    int total = 0;
    for (int g0 = 0; g0 < x; g0 += kApTrialThreads) {
        const int g = g0 + tid;
        const bool e = g < x && rank[base + g] == 0 && cnt[base + g] >= s;
        const unsigned bal = __ballot_sync(0xffffffffu, e);
        if (lane == 0) s_w[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {
            const int v = s_w[lane];
            int sc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, sc, o);
                if (lane >= o) sc += u;
            }
            s_w[lane] = sc - v;
            if (lane == 31) s_w[32] = sc;
        }
        __syncthreads();
        if (e) {
            const int q = total + s_w[warp] + __popc(bal & ((1u << lane) - 1u));
            if (q < kApMaxBuckets) {
                s_key[q] = keys[base + g];
                s_g[q] = g;
            }
        }
        total += s_w[32];
        __syncthreads();
    }
    if (total > kApMaxBuckets) {
        if (tid == 0) {
            atomicExch(err, 1);
            nb[blockIdx.x] = 0;
            nm[blockIdx.x] = 0;
        }
        return;
    }
    // bitonic sort by key (keys of distinct buckets differ; k <= 15 keeps every key
    // below the padding value) over the next power of two
    int n2 = 1;
    while (n2 < total) n2 <<= 1;
    for (int q = total + tid; q < n2; q += kApTrialThreads) s_key[q] = 0xFFFFFFFFu;
    __syncthreads();
    for (int size = 2; size <= n2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int q = tid; q < n2; q += kApTrialThreads) {
                const int p = q ^ stride;
                if (p > q) {
                    const bool up = (q & size) == 0;
                    if ((s_key[q] > s_key[p]) == up) {
                        const uint32_t tk = s_key[q]; s_key[q] = s_key[p]; s_key[p] = tk;
                        const int32_t tg = s_g[q]; s_g[q] = s_g[p]; s_g[p] = tg;
                    }
                }
            }
            __syncthreads();
        }
    }
    // member offsets in key order (one warp: a running prefix over the list)
    if (warp == 0) {
        int run = 0;
        for (int q0 = 0; q0 < total; q0 += 32) {
            const int q = q0 + lane;
            const int v = q < total ? cnt[base + s_g[q]] : 0;
            int sc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, sc, o);
                if (lane >= o) sc += u;
            }
            if (q < total) {
                list[(int64_t)blockIdx.x * kApMaxBuckets + q] = make_uint2(s_key[q], (uint32_t)s_g[q]);
                lsize[(int64_t)blockIdx.x * kApMaxBuckets + q] = v;
                loff[(int64_t)blockIdx.x * kApMaxBuckets + q] = run + sc - v;
            }
            run += __shfl_sync(0xffffffffu, sc, 31);
        }
        if (lane == 0) {
            nb[blockIdx.x] = total;
            nm[blockIdx.x] = run;
        }
    }
}

// Exclusive scan of the per-trial counts (one CTA): candidate and member
// offsets, the totals, and cand_off[C] = total members when it fits.
__global__ void __launch_bounds__(1024) ap_scan_kernel(const int32_t *__restrict__ nb,
                                                       const int32_t *__restrict__ nm, int n,
                                                       int64_t *__restrict__ cbase,
                                                       int64_t *__restrict__ mbase,
                                                       int64_t *__restrict__ totals,
                                                       int64_t cap_cand,
                                                       int64_t *__restrict__ cand_off) {
    __shared__ long long s_a[1024], s_b[1024];
    const int tid = threadIdx.x;
    const int chunk = (n + 1023) / 1024;
    const int lo = min(tid * chunk, n), hi = min(lo + chunk, n);
    long long a = 0, b = 0;
    for (int e = lo; e < hi; ++e) { a += nb[e]; b += nm[e]; }
    s_a[tid] = a;
    s_b[tid] = b;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const long long va = tid >= o ? s_a[tid - o] : 0, vb = tid >= o ? s_b[tid - o] : 0;
        __syncthreads();
        s_a[tid] += va;
        s_b[tid] += vb;
        __syncthreads();
    }
    long long pa = s_a[tid] - a, pb = s_b[tid] - b;
    for (int e = lo; e < hi; ++e) {
        cbase[e] = pa;
        mbase[e] = pb;
        pa += nb[e];
        pb += nm[e];
    }
    if (tid == 1023) {
        totals[0] = s_a[1023];
        totals[1] = s_b[1023];
        if (s_a[1023] <= cap_cand) cand_off[s_a[1023]] = s_b[1023];
    }
}

// Candidate table of trial blockIdx.y; lead_off[trial][g] = member offset of
// the bucket whose first l-mer is g.
__global__ void ap_write_kernel(const uint2 *__restrict__ list, const int32_t *__restrict__ lsize,
                                const int32_t *__restrict__ loff, const int32_t *__restrict__ nb,
                                const int64_t *__restrict__ cbase,
                                const int64_t *__restrict__ mbase, int x, int64_t trial_begin,
                                int64_t cap_cand, int32_t *__restrict__ cand_trial,
                                uint32_t *__restrict__ cand_key, int32_t *__restrict__ cand_cnt,
                                int64_t *__restrict__ cand_off, int64_t *__restrict__ lead_off) {
    const int tr = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb[tr]) return;
    const int64_t q = (int64_t)tr * kApMaxBuckets + i;
    const uint2 e = list[q];
    const int64_t off = mbase[tr] + loff[q];
    const int64_t ci = cbase[tr] + i;
    if (ci < cap_cand) {
        cand_trial[ci] = (int32_t)(trial_begin + tr);
        cand_key[ci] = e.x;
        cand_cnt[ci] = lsize[q];
        cand_off[ci] = off;
    }
    lead_off[(int64_t)tr * x + e.y] = off;
}

__global__ void ap_members_kernel(const int32_t *__restrict__ cnt, const int32_t *__restrict__ rank,
                                  const int32_t *__restrict__ lead,
                                  const int64_t *__restrict__ lead_off, int x, int s,
                                  int64_t cap_members, int32_t *__restrict__ members) {
    const int64_t base = (int64_t)blockIdx.y * x;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= x || cnt[base + g] < s) return;
    const int64_t p = lead_off[base + lead[base + g]] + rank[base + g];
    if (p < cap_members) members[p] = g;
}

constexpr int kSortMax = 16384;  // l-mers per trial the sort path holds in shared memory

// Block-wide exclusive scan of two counters (1024 threads); also returns totals.
__device__ __forceinline__ void se_scan2(int a, int b, int &ea, int &eb, int &ta, int &tb) {
    __shared__ int s_a[32], s_b[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ua = __shfl_up_sync(0xffffffffu, ia, o), ub = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) { ia += ua; ib += ub; }
    }
    if (lane == 31) { s_a[warp] = ia; s_b[warp] = ib; }
    __syncthreads();
    if (warp == 0) {
        int va = s_a[lane], vb = s_b[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ua = __shfl_up_sync(0xffffffffu, va, o), ub = __shfl_up_sync(0xffffffffu, vb, o);
            if (lane >= o) { va += ua; vb += ub; }
        }
        s_a[lane] = va;
        s_b[lane] = vb;
    }
    __syncthreads();
    const int pa = warp > 0 ? s_a[warp - 1] : 0, pb = warp > 0 ? s_b[warp - 1] : 0;
    ea = pa + ia - a;
    eb = pb + ib - b;
    ta = s_a[31];
    tb = s_b[31];
    __syncthreads();
}

// One CTA per trial: (key << 32 | l-mer) pairs sorted ascending in shared
// memory (p2 = the power of two >= x; padding sorts last), written to
// sorted[trial][x]; nb / nm = the trial's runs of >= s equal keys and their
// l-mers.
__global__ void __launch_bounds__(1024) se_sort_kernel(const uint32_t *__restrict__ keys, int x,
                                                       int p2, int s,
                                                       unsigned long long *__restrict__ sorted,
                                                       int32_t *__restrict__ nb,
                                                       int32_t *__restrict__ nm) {
    extern __shared__ unsigned long long kv[];
    const int tr = blockIdx.x, tid = threadIdx.x;
    const uint32_t *kt = keys + (int64_t)tr * x;
    for (int i = tid; i < p2; i += 1024)
        kv[i] = i < x ? ((unsigned long long)kt[i] << 32) | (unsigned)i : ~0ull;
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < p2; i += 1024) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long a = kv[i], b = kv[ixj];
                    if ((a > b) == ((i & k) == 0)) {
                        kv[i] = b;
                        kv[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    int lnb = 0, lnm = 0;
    for (int i = tid; i < x; i += 1024) {
        const uint32_t key = (uint32_t)(kv[i] >> 32);
        if (i > 0 && (uint32_t)(kv[i - 1] >> 32) == key) continue;  // not a run start
        int len = 1;
        while (i + len < x && (uint32_t)(kv[i + len] >> 32) == key) ++len;
        if (len >= s) { ++lnb; lnm += len; }
    }
    int ea, eb, ta, tb;
    se_scan2(lnb, lnm, ea, eb, ta, tb);
    if (tid == 0) { nb[tr] = ta; nm[tr] = tb; }
    for (int i = tid; i < x; i += 1024) sorted[(int64_t)tr * x + i] = kv[i];
}

// One CTA per trial: the enriched runs of its sorted pairs in key order ->
// candidate table rows at cbase[trial] and member lists at mbase[trial] (ids
// ascending within a run, as the pairs are sorted by (key, l-mer)).
__global__ void __launch_bounds__(1024) se_write_kernel(
    const unsigned long long *__restrict__ sorted, int x, int s, const int64_t *__restrict__ cbase,
    const int64_t *__restrict__ mbase, int64_t trial_begin, int64_t cap_cand,
    int64_t cap_members, int32_t *__restrict__ cand_trial, uint32_t *__restrict__ cand_key,
    int32_t *__restrict__ cand_cnt, int64_t *__restrict__ cand_off,
    int32_t *__restrict__ members) {
    const int tr = blockIdx.x, tid = threadIdx.x;
    const unsigned long long *kt = sorted + (int64_t)tr * x;
    const int chunk = (x + 1023) / 1024;
    const int c0 = min(tid * chunk, x), c1 = min(c0 + chunk, x);
    auto run_len = [&](int i, uint32_t key) {
        int len = 1;
        while (i + len < x && (uint32_t)(kt[i + len] >> 32) == key) ++len;
        return len;
    };
    int cnt = 0, msum = 0;
    for (int i = c0; i < c1; ++i) {
        const uint32_t key = (uint32_t)(kt[i] >> 32);
        if (i > 0 && (uint32_t)(kt[i - 1] >> 32) == key) continue;
        const int len = run_len(i, key);
        if (len >= s) { ++cnt; msum += len; }
    }
    int rb, rm, ta, tb;
    se_scan2(cnt, msum, rb, rm, ta, tb);
    for (int i = c0; i < c1; ++i) {
        const uint32_t key = (uint32_t)(kt[i] >> 32);
        if (i > 0 && (uint32_t)(kt[i - 1] >> 32) == key) continue;
        const int len = run_len(i, key);
        if (len < s) continue;
        const int64_t ci = cbase[tr] + rb, off = mbase[tr] + rm;
        if (ci < cap_cand) {
            cand_trial[ci] = (int32_t)(trial_begin + tr);
            cand_key[ci] = key;
            cand_cnt[ci] = len;
            cand_off[ci] = off;
        }
        for (int q = 0; q < len; ++q)
            if (off + q < cap_members) members[off + q] = (int32_t)(kt[i + q] & 0xFFFFFFFFu);
        ++rb;
        rm += len;
    }
}

}  // namespace
}  // namespace proj

using namespace proj;

namespace proj {

int run_allpairs(const uint32_t *packed, const uint8_t *codes, int alphabet, const Layout &L,
                 int k, int s, uint64_t seed, int64_t trial_begin, int64_t n_trials,
                 int64_t cap_cand, int64_t cap_members, int32_t *cand_trial_dev,
                 uint32_t *cand_key_dev, int32_t *cand_cnt_dev, int64_t *cand_off_dev,
                 int32_t *members_dev, int64_t *totals_dev, cudaStream_t st) {
    if (n_trials == 0) {
        PROJ_CUDA_TRY(cudaMemsetAsync(totals_dev, 0, 2 * sizeof(int64_t), st));
        PROJ_CUDA_TRY(cudaMemsetAsync(cand_off_dev, 0, sizeof(int64_t), st));
        return PROJ_OK;
    }
    const int64_t T = n_trials, x = L.x;
    const int t = L.t, l = L.l;
    PROJ_REQUIRE(T * x < ((int64_t)1 << 31), "n_trials * x must stay below 2^31 per call");
    DevBuf scratch;
    const size_t per = (size_t)T * x;
    const size_t bytes = per * (4 + 4 + 4 + 4 + 8) + (size_t)T * kApMaxBuckets * (8 + 4 + 4) +
                         (size_t)T * (4 + 4 + 8 + 8) + 64;
    PROJ_TRY(scratch.alloc(bytes, st));
    uint8_t *p = scratch.as<uint8_t>();
    int64_t *lead_off = reinterpret_cast<int64_t *>(p); p += per * 8;
    uint2 *list = reinterpret_cast<uint2 *>(p); p += (size_t)T * kApMaxBuckets * 8;
    int64_t *cbase = reinterpret_cast<int64_t *>(p); p += (size_t)T * 8;
    int64_t *mbase = reinterpret_cast<int64_t *>(p); p += (size_t)T * 8;
    uint32_t *keys = reinterpret_cast<uint32_t *>(p); p += per * 4;
    int32_t *cnt = reinterpret_cast<int32_t *>(p); p += per * 4;
    int32_t *rank = reinterpret_cast<int32_t *>(p); p += per * 4;
    int32_t *lead = reinterpret_cast<int32_t *>(p); p += per * 4;
    int32_t *lsize = reinterpret_cast<int32_t *>(p); p += (size_t)T * kApMaxBuckets * 4;
    int32_t *loff = reinterpret_cast<int32_t *>(p); p += (size_t)T * kApMaxBuckets * 4;
    int32_t *nb = reinterpret_cast<int32_t *>(p); p += (size_t)T * 4;
    int32_t *nm = reinterpret_cast<int32_t *>(p); p += (size_t)T * 4;
    int *err = reinterpret_cast<int *>(p);
    PROJ_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    const dim3 grid_x((unsigned)((x + kApThreads - 1) / kApThreads), (unsigned)T);
    {
        TraceSpan ts_("allpairs", st);
        if (alphabet == 20)
            ap_keys_aa_kernel<<<grid_x, kApThreads, 0, st>>>(codes, L.seq_off_dev(), L.lmer_off_dev(),
                                                             t, l, k, (int)x, seed, trial_begin, keys);
        else
            ap_keys_kernel<<<grid_x, kApThreads, 0, st>>>(packed, L.nwords, L.seq_off_dev(),
                                                          L.lmer_off_dev(), t, l, k, (int)x, seed,
                                                          trial_begin, keys);
    }
    PROJ_LAUNCH_CHECK("ap_keys_kernel");
    if (alphabet == 20 && x <= kSortMax) {  // sort path
        int p2 = 2;
        while (p2 < x) p2 <<= 1;
        unsigned long long *sorted = reinterpret_cast<unsigned long long *>(lead_off);
        const size_t smem = (size_t)p2 * 8;
        PROJ_CUDA_TRY(cudaFuncSetAttribute(se_sort_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        {
            TraceSpan ts_("enrich_sort", st);
            se_sort_kernel<<<(unsigned)T, 1024, smem, st>>>(keys, (int)x, p2, s, sorted, nb, nm);
        }
        PROJ_LAUNCH_CHECK("se_sort_kernel");
        {
            TraceSpan ts_("enrich_sort", st);
            ap_scan_kernel<<<1, 1024, 0, st>>>(nb, nm, (int)T, cbase, mbase, totals_dev, cap_cand,
                                               cand_off_dev);
        }
        PROJ_LAUNCH_CHECK("ap_scan_kernel");
        {
            TraceSpan ts_("enrich_sort", st);
            se_write_kernel<<<(unsigned)T, 1024, 0, st>>>(sorted, (int)x, s, cbase, mbase,
                                                          trial_begin, cap_cand, cap_members,
                                                          cand_trial_dev, cand_key_dev, cand_cnt_dev,
                                                          cand_off_dev, members_dev);
        }
        PROJ_LAUNCH_CHECK("se_write_kernel");
        return PROJ_OK;
    }
    {
        TraceSpan ts_("allpairs", st);
        ap_compare_kernel<<<grid_x, kApThreads, 0, st>>>(keys, (int)x, cnt, rank, lead);
    }
    PROJ_LAUNCH_CHECK("ap_compare_kernel");
    {
        TraceSpan ts_("allpairs", st);
        ap_trial_kernel<<<(unsigned)T, kApTrialThreads, 0, st>>>(keys, cnt, rank, (int)x, s, list,
                                                                lsize, loff, nb, nm, err);
    }
    PROJ_LAUNCH_CHECK("ap_trial_kernel");
    int herr = 0;
    PROJ_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    PROJ_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr) {
        set_error("a trial has more than %d enriched buckets (all-pairs mode limit)", kApMaxBuckets);
        return PROJ_ECAPACITY;
    }
    {
        TraceSpan ts_("allpairs", st);
        ap_scan_kernel<<<1, 1024, 0, st>>>(nb, nm, (int)T, cbase, mbase, totals_dev, cap_cand,
                                           cand_off_dev);
    }
    PROJ_LAUNCH_CHECK("ap_scan_kernel");
    {
        TraceSpan ts_("allpairs", st);
        ap_write_kernel<<<dim3(kApMaxBuckets / 256, (unsigned)T), 256, 0, st>>>(
            list, lsize, loff, nb, cbase, mbase, (int)x, trial_begin, cap_cand, cand_trial_dev,
            cand_key_dev, cand_cnt_dev, cand_off_dev, lead_off);
    }
    PROJ_LAUNCH_CHECK("ap_write_kernel");
    if (cap_members > 0) {
        TraceSpan ts_("allpairs", st);
        ap_members_kernel<<<grid_x, kApThreads, 0, st>>>(cnt, rank, lead, lead_off, (int)x, s,
                                                         cap_members, members_dev);
    }
    PROJ_LAUNCH_CHECK("ap_members_kernel");
    return PROJ_OK;
}

}  // namespace proj

extern "C" int trial_hash_allpairs(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l,
                                   int k, int s, uint64_t seed, int64_t trial_begin,
                                   int64_t n_trials, int64_t cap_cand, int64_t cap_members,
                                   int32_t *cand_trial_dev, uint32_t *cand_key_dev,
                                   int32_t *cand_cnt_dev, int64_t *cand_off_dev,
                                   int32_t *members_dev, int64_t *totals_dev, void *stream) {
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    PROJ_REQUIRE(packed_dev != nullptr && totals_dev != nullptr && cand_off_dev != nullptr,
                 "packed_dev, cand_off_dev and totals_dev must not be NULL");
    PROJ_REQUIRE(k >= 1 && k <= 15 && k <= l, "need 1 <= k <= min(l, 15)");
    PROJ_REQUIRE(s >= 1, "need s >= 1");
    PROJ_REQUIRE(trial_begin >= 0 && n_trials >= 0 && n_trials <= 65535,
                 "need 0 <= n_trials <= 65535 per call");
    PROJ_REQUIRE(cap_cand >= 0 && cap_members >= 0, "capacities must be >= 0");
    PROJ_REQUIRE(cap_cand == 0 || (cand_trial_dev && cand_key_dev && cand_cnt_dev),
                 "candidate buffers must not be NULL");
    PROJ_REQUIRE(cap_members == 0 || members_dev, "members_dev must not be NULL");
    Layout L;
    PROJ_TRY(make_layout(seq_off, t, l, st, L));
    return run_allpairs(packed_dev, nullptr, 4, L, k, s, seed, trial_begin, n_trials, cap_cand,
                        cap_members, cand_trial_dev, cand_key_dev, cand_cnt_dev, cand_off_dev,
                        members_dev, totals_dev, st);
}
