// EM refinement (Section 5.1, OOPS) with both contractions on the tcgen05
// tensor cores: PROJ_EM_BF16_SPLIT.
//
// The E-step score of candidate c on l-mer j, r(c,j) = sum_p W_c[p][x_{j+p}],
// is the product of the log-odds matrix W [C x 4l] with the one-hot encoding
// X [x x 4l] of the l-mers (exact in BF16).  The M-step counts
// N_c[p][a] = sum_j z(c,j) [x_{j+p} = a] are the product of the posteriors
// Z [C x x] with the same X.  Together they have the shape of attention with
// one-hot keys and values: per sequence a softmax over the starts j.
//
// Work is a list of items, each = (instance, up to 128 candidates of it, a
// range of its sequences); a CTA (128 threads = the 128 lanes of tensor
// memory) takes items in turn from the list (persistent over the list when the
// grid is smaller than it), so one launch serves one motif search or a batch of
// many instances of different t, n and l.  Per tile of NT l-mers of a sequence:
//   1. the CTA writes the one-hot tile X [NT x 4l] to shared memory (from the
//      sequence's packed words, staged in shared memory);
//   2. one thread issues S = W_hi X^T + W_lo X^T (M=128, N=NT, K=16*ceil(4l/16),
//      FP32 accumulation in tensor memory; W split into BF16 hi + lo parts so
//      the product carries ~16 mantissa bits of W);
//   3. thread i reads row i of S, keeps a running maximum and a compensated
//      running sum of 2^(S - max) for its candidate, rescales its row of O when
//      the maximum grows, and writes P = 2^(S - max) as BF16 hi + lo parts;
//   4. one thread issues O += P_hi X + P_lo X (M=128, N=16*ceil(4l/16), K=NT)
//      with X read in MN-major form from the same shared-memory tile.
// At the end of a sequence O / sum is added to the candidate's counts and
// max + log2(sum) to its log-likelihood.  Scores are kept in log2 units
// (W = log2 theta - log2 bg) so the exponentials are exp2.
//
// Every wait on an MMA completion is bounded; when a bound expires the CTA
// stops, records the failure in a device flag (returned as PROJ_ETIMEOUT) and
// frees its tensor memory.
#include <math.h>

#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "em_batch.cuh"
#include "tc.cuh"

namespace proj {
namespace {

constexpr int kTcThreads = 128;
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s per wait on a tensor-core completion

struct EmTcParams {
    const uint32_t *packed;
    int64_t nwords;
    const EmInst *inst;     // [n_inst]
    const EmItem *items;    // [n_items]
    int n_items;
    const float *theta_in;  // [C][stride]
    int stride;             // floats per candidate model (>= 4l of its instance)
    double *part_acc;       // [G][C][stride]; G == 1 when no candidate tile is split
    double *part_ll;        // [G][C]
    int64_t C;
    int mstep;
    int *err;
};

template <int KP, int NT>
struct TcLayout {
    static constexpr int W_BYTES = 128 * KP * 2;  // each of W_hi, W_lo
    static constexpr int X_BYTES = NT * KP * 2;
    static constexpr int P_BYTES = 128 * NT * 2;  // each of P_hi, P_lo
    static constexpr int OFF_WHI = 0;
    static constexpr int OFF_WLO = OFF_WHI + W_BYTES;
    static constexpr int OFF_X = OFF_WLO + W_BYTES;
    static constexpr int OFF_PHI = OFF_X + X_BYTES;
    static constexpr int OFF_PLO = OFF_PHI + P_BYTES;
    static constexpr int SEQ_WORDS = 512;  // staged packed words of one sequence (8K bases)
    static constexpr int OFF_SEQ = OFF_PLO + P_BYTES;
    static constexpr int TOTAL = OFF_SEQ + SEQ_WORDS * 4;
    static constexpr uint32_t TMEM_COLS = (NT + KP <= 128) ? 128u : 256u;
};

__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void kahan(float &sum, float &comp, float v) {
    const float y = v - comp;
    const float s = sum + y;
    comp = (s - sum) - y;
    sum = s;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

template <int KP, int NT>
__global__ void __launch_bounds__(kTcThreads, (KP <= 80 ? 3 : 2)) em_tc_kernel(const EmTcParams P) {
    using LY = TcLayout<KP, NT>;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    uint8_t *sWhi = smem + LY::OFF_WHI, *sWlo = smem + LY::OFF_WLO, *sX = smem + LY::OFF_X;
    uint8_t *sPhi = smem + LY::OFF_PHI, *sPlo = smem + LY::OFF_PLO;
    uint32_t *sSeq = reinterpret_cast<uint32_t *>(smem + LY::OFF_SEQ);

    if (tid == 0) {
        tc::mbar_init(&mbar, 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&tmem_slot, LY::TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = tmem_slot;
    const uint32_t tS = tm, tO = tm + NT;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const uint32_t aWhi = tc::smem_addr(sWhi), aWlo = tc::smem_addr(sWlo);
    const uint32_t aX = tc::smem_addr(sX), aPhi = tc::smem_addr(sPhi), aPlo = tc::smem_addr(sPlo);
    constexpr uint32_t IDESC_S = tc::idesc_bf16(128, NT);
    uint32_t phase = 0;
    bool abort = false;

    for (int it = blockIdx.x; it < P.n_items && !abort; it += gridDim.x) {
        const EmItem item = P.items[it];
        const EmInst in = P.inst[item.inst];
        const int l = in.l, L4 = 4 * l;
        const int kq = (L4 + 15) / 16;  // K steps of the score MMA = N / 16 of the count MMA
        const uint32_t idesc_o = tc::idesc_bf16(128, 16 * kq, true);
        const int64_t c = item.c0 + tid;
        const bool valid = tid < item.nc;

        // W_c = log2 theta_c - log2 bg in FP32 (~2^-23 relative, far below the
        // 2^-16 of the BF16 hi + lo pair), split into BF16 hi + lo (row tid)
        __syncthreads();  // the previous item's MMAs and reads are complete
        float lbg[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) lbg[a] = log2f((float)in.bg[a]);
        for (int k8 = 0; k8 < KP; k8 += 8) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
                float h2[2], l2[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int k = k8 + q + u;
                    float w = 0.f;
                    if (valid && k < L4) w = log2f(__ldg(P.theta_in + c * P.stride + k)) - lbg[k & 3];
                    const float h = __bfloat162float(__float2bfloat16_rn(w));
                    h2[u] = h;
                    l2[u] = w - h;
                }
                hi[q / 2] = pack_bf16(h2[0], h2[1]);
                lo[q / 2] = pack_bf16(l2[0], l2[1]);
            }
            *reinterpret_cast<uint4 *>(sWhi + tc::kmajor_off(tid, k8, KP)) =
                make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(sWlo + tc::kmajor_off(tid, k8, KP)) =
                make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        tc::fence_async_smem();

        // this item's normalised counts of candidate c, summed over its sequences
        float tot[KP];
#pragma unroll
        for (int q = 0; q < KP; ++q) tot[q] = 0.f;
        double ll = 0.0;

        for (int i = item.seq_lo; i < item.seq_hi && !abort; ++i) {
            const int64_t base = in.seq_off[i];
            const int n_i = in.seq_off[i + 1] - in.seq_off[i];
            const int ns = n_i - l + 1;
            float m = -INFINITY, Ssum = 0.f, Scmp = 0.f;
            bool first = true;
            // packed words covering this sequence (+2 for the 64-bit windows)
            const int64_t w_first = base >> 4;
            const int nw_seq = (int)(((base + n_i + 15) >> 4) - w_first) + 2;
            const bool staged = nw_seq <= LY::SEQ_WORDS;
            __syncthreads();  // the previous sequence's words are no longer read
            if (staged)
                for (int w = tid; w < nw_seq; w += kTcThreads)
                    sSeq[w] = (w_first + w) < P.nwords ? __ldg(P.packed + w_first + w) : 0u;
            __syncthreads();
            for (int j0 = 0; j0 < ns; j0 += NT) {
                const int nvalid = min(NT, ns - j0);
                // 1. one-hot tile X[j][p*4+a] = [x_{j0+j+p} = a]: thread (j, half) writes
                //    16-byte chunks kb (two positions each, BF16 1.0 = 0x3F80 in the slot of
                //    the base's code) of row j from one 64-bit window
                static_assert(kTcThreads % NT == 0, "rows must divide the CTA");
                {
                    constexpr int kSplit = kTcThreads / NT;  // threads per row
                    constexpr int kChunks = KP / 8;
                    const int j = tid % NT, part = tid / NT;
                    const bool row_ok = j < nvalid;
                    uint64_t win = 0;
                    if (row_ok)
                        win = staged ? window64(sSeq, nw_seq, base + j0 + j - (w_first << 4))
                                     : window64(P.packed, P.nwords, base + j0 + j);
#pragma unroll
                    for (int kb = part; kb < kChunks; kb += kSplit) {
                        uint32_t w0 = 0u, w1 = 0u, w2 = 0u, w3 = 0u;
                        const int p0 = 2 * kb, p1 = 2 * kb + 1;
                        if (row_ok && p0 < l) {
                            const uint32_t code = (uint32_t)(win >> (2 * p0)) & 3u;
                            const uint32_t v = 0x3F80u << (16 * (code & 1u));
                            if (code >> 1) w1 = v; else w0 = v;
                        }
                        if (row_ok && p1 < l) {
                            const uint32_t code = (uint32_t)(win >> (2 * p1)) & 3u;
                            const uint32_t v = 0x3F80u << (16 * (code & 1u));
                            if (code >> 1) w3 = v; else w2 = v;
                        }
                        *reinterpret_cast<uint4 *>(sX + tc::kmajor_off(j, 8 * kb, KP)) =
                            make_uint4(w0, w1, w2, w3);
                    }
                }
                tc::fence_async_smem();
                __syncthreads();
                // 2. S = W_hi X^T + W_lo X^T
                if (tid == 0) {
                    tc::fence_after_sync();
                    for (int s = 0; s < kq; ++s)
                        tc::mma_bf16(tS, tc::sdesc(aWhi + 256 * s, 128, KP * 16),
                                     tc::sdesc(aX + 256 * s, 128, KP * 16), IDESC_S, s > 0);
                    for (int s = 0; s < kq; ++s)
                        tc::mma_bf16(tS, tc::sdesc(aWlo + 256 * s, 128, KP * 16),
                                     tc::sdesc(aX + 256 * s, 128, KP * 16), IDESC_S, 1);
                    tc::mma_commit(&mbar);
                }
                bool ok = tc::mbar_wait(&mbar, phase, kWaitNs);
                phase ^= 1u;
                abort = __syncthreads_or(!ok);
                if (abort) break;
                tc::fence_after_sync();
                // 3. P = 2^(S - m) with m a reference near the row maximum: the exact
                //    maximum of the first tile of a sequence, then kept until a tile
                //    holds a score more than 20 above it (P > 2^20); only then is the
                //    maximum recomputed and the row's O and sum rescaled.  Each 32-column
                //    chunk is summed as a tree and the chunk sums are added with
                //    compensation.  The tensor-memory accesses are .sync.aligned, so
                //    every decision that guards them is taken per warp.
                const bool full = nvalid == NT;  // only a sequence's last tile is ragged
                bool redo = first;
                for (int pass = 0; pass < 2; ++pass) {
                    if (redo) {
                        float tmax = -INFINITY;
#pragma unroll
                        for (int c0 = 0; c0 < NT; c0 += 32) {
                            float v[32];
                            tc::tmem_ld32(tS + lane_base + c0, v);
                            float mx[8];
#pragma unroll
                            for (int q = 0; q < 8; ++q) mx[q] = -INFINITY;
                            if (full) {
#pragma unroll
                                for (int q = 0; q < 32; ++q) mx[q & 7] = fmaxf(mx[q & 7], v[q]);
                            } else {
#pragma unroll
                                for (int q = 0; q < 32; ++q)
                                    if (c0 + q < nvalid) mx[q & 7] = fmaxf(mx[q & 7], v[q]);
                            }
#pragma unroll
                            for (int q = 0; q < 8; ++q) tmax = fmaxf(tmax, mx[q]);
                        }
                        const bool grow = tmax > m;
                        const float sc = grow ? ex2(m - tmax) : 1.f;  // 0 when m = -inf
                        if (grow) {
                            Ssum *= sc;
                            Scmp *= sc;
                            m = tmax;
                        }
                        if (P.mstep && !first && __any_sync(0xffffffffu, grow)) {
#pragma unroll
                            for (int c0 = 0; c0 < KP; c0 += 16) {
                                if (c0 < 16 * kq) {
                                    float v[16];
                                    tc::tmem_ld16(tO + lane_base + c0, v);
#pragma unroll
                                    for (int q = 0; q < 16; ++q) v[q] *= sc;
                                    tc::tmem_st16(tO + lane_base + c0, v);
                                }
                            }
                        }
                    }
                    float add = 0.f;  // this tile's sum, chunk by chunk
                    bool big = false;
#pragma unroll
                    for (int c0 = 0; c0 < NT; c0 += 32) {
                        float v[32];
                        tc::tmem_ld32(tS + lane_base + c0, v);
                        if (full) {
#pragma unroll
                            for (int q = 0; q < 32; ++q) v[q] = ex2(v[q] - m);
                        } else {
#pragma unroll
                            for (int q = 0; q < 32; ++q) v[q] = (c0 + q < nvalid) ? ex2(v[q] - m) : 0.f;
                        }
                        float part[16];
#pragma unroll
                        for (int q = 0; q < 16; ++q) part[q] = v[2 * q] + v[2 * q + 1];
#pragma unroll
                        for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
                            for (int q = 0; q < w; ++q) part[q] += part[q + w];
                        add += part[0];
                        big |= part[0] > 1048576.f;  // some score > m + 20 (or NaN-free inf)
                        if (P.mstep) {
                            uint32_t hi[16], lo[16];
#pragma unroll
                            for (int q = 0; q < 16; ++q) {
                                const uint32_t h = pack_bf16(v[2 * q], v[2 * q + 1]);
                                const float h0 = __uint_as_float(h << 16);
                                const float h1 = __uint_as_float(h & 0xFFFF0000u);
                                hi[q] = h;
                                lo[q] = pack_bf16(v[2 * q] - h0, v[2 * q + 1] - h1);
                            }
#pragma unroll
                            for (int b = 0; b < 4; ++b) {
                                *reinterpret_cast<uint4 *>(sPhi + tc::kmajor_off(tid, c0 + 8 * b, NT)) =
                                    make_uint4(hi[4 * b], hi[4 * b + 1], hi[4 * b + 2], hi[4 * b + 3]);
                                *reinterpret_cast<uint4 *>(sPlo + tc::kmajor_off(tid, c0 + 8 * b, NT)) =
                                    make_uint4(lo[4 * b], lo[4 * b + 1], lo[4 * b + 2], lo[4 * b + 3]);
                            }
                        }
                    }
                    redo = __any_sync(0xffffffffu, big) && pass == 0;
                    if (!redo) {
                        kahan(Ssum, Scmp, add);
                        break;
                    }
                }
                tc::fence_before_sync();
                if (P.mstep) {
                    // 4. O += P_hi X + P_lo X
                    tc::fence_async_smem();
                    __syncthreads();
                    if (tid == 0) {
                        tc::fence_after_sync();
#pragma unroll
                        for (int s = 0; s < NT / 16; ++s)
                            tc::mma_bf16(tO, tc::sdesc(aPhi + 256 * s, 128, NT * 16),
                                         tc::sdesc(aX + s * 2 * KP * 16, KP * 16, 128), idesc_o,
                                         (s > 0 || !first) ? 1u : 0u);
#pragma unroll
                        for (int s = 0; s < NT / 16; ++s)
                            tc::mma_bf16(tO, tc::sdesc(aPlo + 256 * s, 128, NT * 16),
                                         tc::sdesc(aX + s * 2 * KP * 16, KP * 16, 128), idesc_o, 1u);
                        tc::mma_commit(&mbar);
                    }
                    ok = tc::mbar_wait(&mbar, phase, kWaitNs);
                    phase ^= 1u;
                    abort = __syncthreads_or(!ok);
                    if (abort) break;
                    tc::fence_after_sync();
                } else {
                    __syncthreads();  // every row of S is read before the next tile rewrites it
                }
                first = false;
            }
            if (abort) break;
            const float Sf = Ssum - Scmp;
            ll += (double)((m + log2f(Sf)) * 0.69314718f - logf((float)ns));
            if (P.mstep) {
                const float inv = 1.f / Sf;
#pragma unroll
                for (int c0 = 0; c0 < KP; c0 += 16) {
                    if (c0 < 16 * kq) {
                        float v[16];
                        tc::tmem_ld16(tO + lane_base + c0, v);
#pragma unroll
                        for (int q = 0; q < 16; ++q) tot[c0 + q] += v[q] * inv;
                    }
                }
                tc::fence_before_sync();
                __syncthreads();  // O is read before the next sequence restarts it
            }
        }
        if (abort) break;
        if (valid) {
            P.part_ll[(int64_t)item.g * P.C + c] = ll;
            if (P.mstep) {
                double *dst = P.part_acc + ((int64_t)item.g * P.C + c) * P.stride;
#pragma unroll
                for (int q = 0; q < KP; ++q)
                    if (q < L4) dst[q] = (double)tot[q];
            }
        }
    }
    if (abort) {
        if (tid == 0) atomicExch(P.err, 1);
        // let any MMA still in flight finish (bounded) before freeing its memory:
        // the phase that was being waited for has parity phase ^ 1
        tc::mbar_wait(&mbar, phase ^ 1u, kWaitNs);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tm, LY::TMEM_COLS);
    }
}

// M-step theta = (sum_g counts + pseudocount) / (t + 4 pseudocount) and the
// log-likelihood sum over the G sequence groups, in group order.
__global__ void em_tc_reduce_kernel(const double *__restrict__ part_acc,
                                    const double *__restrict__ part_ll, int G, int64_t C,
                                    int stride, const EmInst *__restrict__ inst, int n_inst,
                                    float beta, int mstep, float *__restrict__ theta_out,
                                    double *__restrict__ ll_out) {
    // one thread per (candidate, model entry); C * stride < 2^31 (checked by the host)
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t width = mstep ? (uint32_t)stride : 1u;
    if ((int64_t)idx >= C * width) return;
    const uint32_t c = idx / width, q = idx - c * width;
    int lo = 0, hi = n_inst - 1;  // instance of candidate c
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (inst[mid].cand_begin <= (int64_t)c) lo = mid; else hi = mid - 1;
    }
    if (mstep && (int)q < 4 * inst[lo].l) {
        double s = 0.0;
        for (int g = 0; g < G; ++g) s += part_acc[((int64_t)g * C + c) * stride + q];
        theta_out[idx] = (float)((s + (double)beta) / ((double)inst[lo].t + 4.0 * (double)beta));
    }
    if (q == 0) {
        double s = 0.0;
        for (int g = 0; g < G; ++g) s += part_ll[(int64_t)g * C + c];
        ll_out[c] = s;
    }
}

template <int KP, int NT>
int launch_tc(const EmTcParams &P, int grid, cudaStream_t st) {
    using LY = TcLayout<KP, NT>;
    PROJ_CUDA_TRY(cudaFuncSetAttribute(em_tc_kernel<KP, NT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, LY::TOTAL));
    {
        TraceSpan ts_("em_tc", st);
        em_tc_kernel<KP, NT><<<grid, kTcThreads, LY::TOTAL, st>>>(P);
    }
    PROJ_LAUNCH_CHECK("em_tc_kernel");
    return PROJ_OK;
}

template <int KP>
int ctas_per_sm_kp() {
    using LY = TcLayout<KP, 64>;
    const int by_smem = 228 * 1024 / (LY::TOTAL + 1024 + 128);
    const int by_tmem = 512 / (int)LY::TMEM_COLS;
    return std::max(1, std::min(by_smem, by_tmem));
}

int ctas_per_sm(int kp) {
    switch (kp) {
        case 16: return ctas_per_sm_kp<16>();
        case 32: return ctas_per_sm_kp<32>();
        case 48: return ctas_per_sm_kp<48>();
        case 64: return ctas_per_sm_kp<64>();
        case 80: return ctas_per_sm_kp<80>();
        case 96: return ctas_per_sm_kp<96>();
        case 112: return ctas_per_sm_kp<112>();
        default: return ctas_per_sm_kp<128>();
    }
}

int dispatch(int kp, const EmTcParams &P, int grid, cudaStream_t st) {
    switch (kp) {
        case 16: return launch_tc<16, 64>(P, grid, st);
        case 32: return launch_tc<32, 64>(P, grid, st);
        case 48: return launch_tc<48, 64>(P, grid, st);
        case 64: return launch_tc<64, 64>(P, grid, st);
        case 80: return launch_tc<80, 64>(P, grid, st);
        case 96: return launch_tc<96, 64>(P, grid, st);
        case 112: return launch_tc<112, 64>(P, grid, st);
        default: return launch_tc<128, 64>(P, grid, st);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Work plan and autotuning.  A schedule is (ctas, g_target): CTAs per SM of
// the persistent grid (<= what shared memory and registers allow) and how
// many work items per CTA slot the sequence-group split aims for when there
// are few candidate tiles.  The first search of each shape class times one
// E-step launch of every candidate schedule on its own data and keeps the
// fastest (per process); PROJ_AUTOTUNE=0 turns this off (default schedule).
// ---------------------------------------------------------------------------
namespace {

struct Sched { int ctas, g_target; };
const Sched kScheds[] = {{3, 2}, {3, 1}, {3, 4}, {2, 2}, {2, 4}, {1, 4}};
constexpr Sched kDefaultSched = {3, 2};

std::mutex g_tune_mu;
std::map<uint64_t, Sched> g_tuned;

uint64_t shape_key(int kp, int64_t C, int tmin, int64_t lmers) {
    int cb = 0, xb = 0;
    while (((int64_t)1 << cb) < C) ++cb;
    while (((int64_t)1 << xb) < lmers) ++xb;
    return ((uint64_t)kp << 48) | ((uint64_t)cb << 40) | ((uint64_t)std::min(tmin, 65535) << 16) |
           (uint64_t)xb;
}

}  // namespace

int em_tc_plan(const std::vector<EmInstHost> &insts, std::vector<EmItem> &items, int &G,
               int ctas, int g_target) {
    // split each instance's candidates into tiles of 128; when there are too
    // few tiles for g_target items per CTA slot, split the sequences into G groups
    int kp = 16;
    int64_t tiles = 0;
    for (const EmInstHost &h : insts) {
        kp = std::max(kp, 16 * ((4 * h.l + 15) / 16));
        tiles += (h.C + kTcThreads - 1) / kTcThreads;
    }
    const int64_t slots = (int64_t)sm_count() * std::min(ctas, ctas_per_sm(kp));
    int tmin = 1 << 30;
    for (const EmInstHost &h : insts) tmin = std::min(tmin, h.t);
    G = 1;
    if (tiles > 0 && tiles < g_target * slots)
        G = (int)std::min<int64_t>(std::max(1, tmin), (g_target * slots + tiles - 1) / tiles);
    items.clear();
    for (size_t ii = 0; ii < insts.size(); ++ii) {
        const EmInstHost &h = insts[ii];
        for (int64_t c0 = 0; c0 < h.C; c0 += kTcThreads)
            for (int g = 0; g < G; ++g) {
                EmItem it;
                it.c0 = h.cand_begin + c0;
                it.nc = (int)std::min<int64_t>(kTcThreads, h.C - c0);
                it.inst = (int)ii;
                it.seq_lo = (int)((int64_t)h.t * g / G);
                it.seq_hi = (int)((int64_t)h.t * (g + 1) / G);
                it.g = g;
                items.push_back(it);
            }
    }
    return kp;
}

int em_tc_prepare(const uint32_t *packed, int64_t nwords, const std::vector<EmInstHost> &insts,
                  const EmInst *inst_dev, const float *theta0, int64_t C, int stride,
                  EmTcRun &run, cudaStream_t st) {
    run.C = C;
    run.stride = stride;
    run.n_inst = (int)insts.size();
    run.inst_dev = inst_dev;
    run.packed = packed;
    run.nwords = nwords;
    run.theta0 = theta0;
    if (C == 0) return PROJ_OK;
    PROJ_REQUIRE(C * (int64_t)stride < ((int64_t)1 << 31), "too many candidate model entries");
    int tmin = 1 << 30;
    int64_t lmers = 0;
    int kp = 16;
    for (const EmInstHost &h : insts) {
        tmin = std::min(tmin, h.t);
        lmers += h.lmers;
        kp = std::max(kp, 16 * ((4 * h.l + 15) / 16));
    }
    PROJ_REQUIRE(kp <= 128, "l above 32 is not supported");
    const uint64_t key = shape_key(kp, C, tmin, lmers);
    Sched sched = kDefaultSched;
    bool known = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) { sched = it->second; known = true; }
    }
    const char *env = getenv("PROJ_AUTOTUNE");
    bool tune = !known && !(env && env[0] == '0');
    // PROJ_EM_SCHED="ctas,g_target" forces one schedule (no tuning, no cache)
    if (const char *fs = getenv("PROJ_EM_SCHED")) {
        int c = 0, g = 0;
        if (sscanf(fs, "%d,%d", &c, &g) == 2 && c >= 1 && c <= 3 && g >= 1 && g <= 8) {
            sched = {c, g};
            tune = false;
        }
    }

    // buffers sized for the largest G any candidate schedule may pick
    int Gmax = 1;
    std::vector<EmItem> items;
    for (const Sched &sc : kScheds) {
        int G = 1;
        em_tc_plan(insts, items, G, sc.ctas, sc.g_target);
        Gmax = std::max(Gmax, G);
    }
    PROJ_TRY(run.part.alloc((size_t)Gmax * C * (stride + 1) * sizeof(double), st));
    PROJ_TRY(run.tmp.alloc((size_t)C * stride * sizeof(float), st));
    PROJ_TRY(run.flag.alloc(sizeof(int), st));
    PROJ_CUDA_TRY(cudaMemsetAsync(run.flag.as<int>(), 0, sizeof(int), st));

    if (tune) {
        // time one E-step launch per schedule on this data
        PROJ_CUDA_TRY(cudaMemcpyAsync(run.tmp.as<float>(), theta0, (size_t)C * stride * sizeof(float),
                                      cudaMemcpyDeviceToDevice, st));
        cudaEvent_t e0, e1;
        PROJ_CUDA_TRY(cudaEventCreate(&e0));
        PROJ_CUDA_TRY(cudaEventCreate(&e1));
        float best_ms = 1e30f;
        for (const Sched &sc : kScheds) {
            int G = 1;
            const int kpp = em_tc_plan(insts, items, G, sc.ctas, sc.g_target);
            DevBuf ib;
            PROJ_TRY(ib.alloc(items.size() * sizeof(EmItem), st));
            PROJ_CUDA_TRY(cudaMemcpyAsync(ib.as<EmItem>(), items.data(), items.size() * sizeof(EmItem),
                                          cudaMemcpyHostToDevice, st));
            EmTcParams P{};
            P.packed = packed; P.nwords = nwords; P.inst = inst_dev; P.items = ib.as<EmItem>();
            P.n_items = (int)items.size(); P.theta_in = run.tmp.as<float>(); P.stride = stride;
            P.part_ll = run.part.as<double>(); P.part_acc = run.part.as<double>() + (size_t)G * C;
            P.C = C; P.err = run.flag.as<int>(); P.mstep = 0;
            const int grid = (int)std::min<int64_t>((int64_t)items.size(),
                                                    (int64_t)sm_count() * std::min(sc.ctas, ctas_per_sm(kpp)));
            PROJ_CUDA_TRY(cudaEventRecord(e0, st));
            PROJ_TRY(dispatch(kpp, P, grid, st));
            PROJ_CUDA_TRY(cudaEventRecord(e1, st));
            PROJ_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            PROJ_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) { best_ms = ms; sched = sc; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = sched;
    }
    run.kp = em_tc_plan(insts, items, run.G, sched.ctas, sched.g_target);
    run.ctas = sched.ctas;
    PROJ_TRY(run.items.alloc(items.size() * sizeof(EmItem), st));
    PROJ_CUDA_TRY(cudaMemcpyAsync(run.items.as<EmItem>(), items.data(), items.size() * sizeof(EmItem),
                                  cudaMemcpyHostToDevice, st));
    run.n_items = (int)items.size();
    return PROJ_OK;
}

int em_tc_enqueue(EmTcRun &run, int iters, float beta, float *theta_out, double *ll,
                  cudaStream_t st) {
    const int64_t C = run.C;
    if (C == 0) return PROJ_OK;
    const int stride = run.stride, G = run.G;
    PROJ_CUDA_TRY(cudaMemcpyAsync(run.tmp.as<float>(), run.theta0, (size_t)C * stride * sizeof(float),
                                  cudaMemcpyDeviceToDevice, st));
    EmTcParams P{};
    P.packed = run.packed;
    P.nwords = run.nwords;
    P.inst = run.inst_dev;
    P.items = run.items.as<EmItem>();
    P.n_items = run.n_items;
    P.theta_in = run.tmp.as<float>();
    P.stride = stride;
    P.part_ll = run.part.as<double>();
    P.part_acc = run.part.as<double>() + (size_t)G * C;
    P.C = C;
    P.err = run.flag.as<int>();
    const int grid = (int)std::min<int64_t>((int64_t)run.n_items,
                                            (int64_t)sm_count() * std::min(run.ctas, ctas_per_sm(run.kp)));
    for (int it = 0; it <= iters; ++it) {
        P.mstep = it < iters;
        PROJ_TRY(dispatch(run.kp, P, grid, st));
        const int64_t n = P.mstep ? C * stride : C;
        {
            TraceSpan ts_("em_reduce", st);
            em_tc_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                P.part_acc, P.part_ll, G, C, stride, run.inst_dev, run.n_inst, beta, P.mstep,
                run.tmp.as<float>(), ll);
        }
        PROJ_LAUNCH_CHECK("em_tc_reduce_kernel");
    }
    PROJ_CUDA_TRY(cudaMemcpyAsync(theta_out, run.tmp.as<float>(), (size_t)C * stride * sizeof(float),
                                  cudaMemcpyDeviceToDevice, st));
    return PROJ_OK;
}

int em_tc_finish(EmTcRun &run, cudaStream_t st) {
    if (run.C == 0) return PROJ_OK;
    int err = 0;
    PROJ_CUDA_TRY(cudaMemcpyAsync(&err, run.flag.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, st));
    PROJ_CUDA_TRY(cudaStreamSynchronize(st));
    if (err) {
        set_error("a bounded wait for tensor-core completion expired in em_tc_kernel");
        return PROJ_ETIMEOUT;
    }
    return PROJ_OK;
}

int run_em_tc_batch(const uint32_t *packed, int64_t nwords, const std::vector<EmInstHost> &insts,
                    const EmInst *inst_dev, const float *theta0, int64_t C, int stride, int iters,
                    float beta, float *theta_out, double *ll, cudaStream_t st) {
    EmTcRun run;
    if (C == 0) return PROJ_OK;
    PROJ_TRY(em_tc_prepare(packed, nwords, insts, inst_dev, theta0, C, stride, run, st));
    PROJ_TRY(run_as_graph(kGraphEm, st, [&](cudaStream_t cs) {
        return em_tc_enqueue(run, iters, beta, theta_out, ll, cs);
    }));
    return em_tc_finish(run, st);
}

int run_em_tc(const uint32_t *packed, const Layout &L, const double *bg, const float *theta0,
              int64_t C, int iters, float beta, float *theta_out, double *ll, cudaStream_t st) {
    std::vector<EmInstHost> insts(1);
    insts[0].t = L.t;
    insts[0].l = L.l;
    insts[0].C = C;
    insts[0].cand_begin = 0;
    insts[0].lmers = L.x;
    EmInst in{};
    in.seq_off = L.seq_off_dev();
    in.t = L.t;
    in.l = L.l;
    in.bg = bg;
    in.cand_begin = 0;
    DevBuf ib;
    PROJ_TRY(ib.alloc(sizeof(EmInst), st));
    PROJ_CUDA_TRY(cudaMemcpyAsync(ib.as<EmInst>(), &in, sizeof(EmInst), cudaMemcpyHostToDevice, st));
    return run_em_tc_batch(packed, L.nwords, insts, ib.as<EmInst>(), theta0, C, 4 * L.l, iters,
                           beta, theta_out, ll, st);
}

}  // namespace proj

// ---------------------------------------------------------------------------
// projection_selftest_wait: exercises the bounded wait of the tensor-core
// kernels on an mbarrier that nothing arrives on.
// ---------------------------------------------------------------------------
namespace proj {
namespace {

__global__ void selftest_wait_kernel(uint64_t timeout_ns, int *flag) {
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&mbar, 1);
        tc::mbar_fence_init();
    }
    __syncthreads();
    const bool ok = tc::mbar_wait(&mbar, 0u, timeout_ns);  // phase 0 never completes
    if (!__syncthreads_or(!ok) && threadIdx.x == 0) *flag = 2;  // unexpected completion
    if (!ok && threadIdx.x == 0) *flag = 1;
}

}  // namespace
}  // namespace proj

extern "C" int projection_selftest_wait(int64_t timeout_ns, void *stream) {
    using namespace proj;
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    PROJ_REQUIRE(timeout_ns > 0 && timeout_ns <= 2000000000LL, "timeout must be in (0, 2 s]");
    DevBuf flag;
    PROJ_TRY(flag.alloc(sizeof(int), st));
    PROJ_CUDA_TRY(cudaMemsetAsync(flag.as<int>(), 0, sizeof(int), st));
    selftest_wait_kernel<<<1, 64, 0, st>>>((uint64_t)timeout_ns, flag.as<int>());
    PROJ_LAUNCH_CHECK("selftest_wait_kernel");
    int h = 0;
    PROJ_CUDA_TRY(cudaMemcpyAsync(&h, flag.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, st));
    PROJ_CUDA_TRY(cudaStreamSynchronize(st));
    if (h == 1) {
        set_error("bounded wait expired after %lld ns, as requested", (long long)timeout_ns);
        return PROJ_ETIMEOUT;
    }
    set_error("the wait did not expire (flag %d)", h);
    return PROJ_ECUDA;
}
