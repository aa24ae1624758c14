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
// range of its sequences); a CTA (128 candidate rows = the 128 lanes of tensor
// memory) takes items in turn from the list (persistent over the list when the
// grid is smaller than it), so one launch serves one motif search or a batch of
// many instances of different t, n and l.  Per tile of NT l-mers of a sequence
// (NT = 64, or 128 in the four-parts-per-row form of the kernel):
//   1. one thread copies the one-hot tile X [NT x 4l] into shared memory with a
//      bulk asynchronous copy (the tiles depend only on the sequences and are
//      built once per EM run, in the MMA operand layout, by em_xtiles_kernel);
//   2. one lane of the MMA warp issues S = W_hi X^T + W_lo X^T (M=128, N=NT, K=16*ceil(4l/16),
//      FP32 accumulation in tensor memory; W split into BF16 hi + lo parts so
//      the product carries ~16 mantissa bits of W);
//   3. the threads of row i (32 l-mers each) read its scores S, add 2^(S - m) to a
//      compensated running sum for the candidate (m a reference maximum, see
//      below) and write P = 2^(S - m) as BF16 hi + lo parts over their own
//      columns of S in tensor memory;
//   4. one lane of the MMA warp issues O += P_hi X + P_lo X (M=128, N=16*ceil(4l/16), K=NT)
//      with P read from tensor memory and X in MN-major form from the same
//      shared-memory tile.
// The steps of consecutive tiles overlap (two score buffers in tensor memory,
// a ring of four one-hot tiles): the score MMA of tile i+1 and the count MMA
// of tile i-1 run on the tensor core while the CUDA cores work on tile i.
// At the end of a sequence m + log2(sum) goes to the candidate's
// log-likelihood and O / sum to its counts (O read during the next tile).
// Scores are kept in log2 units (W = log2 theta - log2 bg) so the
// exponentials are exp2.
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
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "em_batch.cuh"
#include "tc.cuh"

namespace proj {
namespace {

// A CTA runs 4H softmax warps (H threads per candidate row, each taking 32
// l-mers of a tile of 64H) and one MMA-issuing warp.  H = 2: 64-l-mer tiles,
// 256 tensor-memory columns, two CTAs per SM; H = 4: 128-l-mer tiles (half
// the per-tile synchronisation and MMA issue per l-mer), 512 columns, one CTA.
template <int H> constexpr int soft_threads() { return 128 * H; }
template <int H> constexpr int tc_threads() { return 128 * H + 32; }
constexpr int kTcRows = 128;     // candidates per work item = tensor-memory lanes
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s per wait on a tensor-core completion

struct EmTcParams {
    const uint32_t *packed;
    int64_t nwords;
    const EmInst *inst;     // [n_inst]
    const EmItem *items;    // [n_items]
    int n_items;
    const float *theta_in;  // [C][stride]
    int stride;             // floats per candidate model (>= 4l of its instance)
    float *part_acc;        // [G][C][stride]; G == 1 when no candidate tile is split
    double *part_ll;        // [G][C]
    double *part_zs;        // [G][C] expected number of sites (ZOOPS)
    int64_t C;
    int mstep;
    int G;                  // items per candidate tile (consecutive in the item list)
    float beta;             // pseudocount
    float *theta_out;       // [C][stride] M-step result (may be theta_in: rows are
                            // rewritten only after every item reading them is done)
    double *ll_out;         // [C]
    uint32_t *tile_done;    // [n_items / G] finished items per tile, 0 between launches
    const uint8_t *xt;      // one-hot tiles of every sequence, X_BYTES each
    int *err;
};

constexpr int kNT = 64;  // l-mers per tile and part count H / 2 (N of the score MMA, K of the
                         // count MMA is 64 H)
// Up to this many sequence groups per candidate tile the last item of a tile
// folds the groups' partial results itself; beyond it one CTA would serialise
// too much of that work, and a separate grid-wide kernel does it.
constexpr int kFoldMaxG = 4;

template <int KP, int H>
struct TcLayout {
    static constexpr int NT = kNT * H / 2;          // l-mers per tile
    static constexpr int W_BYTES = 128 * KP * 2;   // each of W_hi, W_lo
    static constexpr int X_BYTES = NT * KP * 2;    // one one-hot tile
    static constexpr int NX = 4;                   // ring of one-hot tiles
    static constexpr int OFF_WHI = 0;
    static constexpr int OFF_WLO = OFF_WHI + W_BYTES;
    static constexpr int OFF_X = OFF_WLO + W_BYTES;
    static constexpr int TOTAL = OFF_X + NX * X_BYTES;
    // two score buffers S[2] (NT columns each; P = 2^(S - m) as BF16 hi + lo
    // replaces S in place) and the count accumulator O (KP)
    static constexpr uint32_t TMEM_COLS = H == 2 ? 256 : 512;
    static_assert(2 * NT + KP <= (int)TMEM_COLS, "tensor-memory budget");
    static constexpr int NCH = KP / 8;                // 8-column chunks of a row
    static constexpr int CPT = (NCH + H - 1) / H;     // chunks per thread of a row (at most)
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

// Walks the l-mer tiles of an item's sequences in order: sequence seq, first
// start j0 of the tile, ns = number of starts of the sequence, base = its
// first base in the packed input.
template <int NT>
struct TileIt {
    int seq, j0, ns;
    int base;  // first base of the sequence (inputs hold < 2^31 bases)
    __device__ __forceinline__ void load(const EmInst &in) {
        base = in.seq_off[seq];
        ns = in.seq_off[seq + 1] - base - in.l + 1;
    }
    __device__ __forceinline__ void start(const EmInst &in, int s0, int) {
        seq = s0;
        j0 = 0;
        load(in);
    }
    __device__ __forceinline__ bool last() const { return j0 + NT >= ns; }
    __device__ __forceinline__ void advance(const EmInst &in, int seq_hi) {
        j0 += NT;
        if (j0 >= ns) {
            ++seq;
            j0 = 0;
            if (seq < seq_hi) load(in);
        }
    }
};

// One-hot tiles X[j][p*4+a] = [x_{j0+j+p} = a] of every sequence (nt rows per
// tile, nt = 64 or 128), in the K-major core-matrix layout the MMAs read (KP
// columns, rows past the sequence's last l-mer zero), one CTA per sequence:
// thread (row j, part) writes every (256/nt)-th 16-byte chunk (two positions
// each, BF16 1.0 = 0x3F80 in the slot of the base's code) of row j, from one
// 64-bit window of the packed sequence.
__global__ void __launch_bounds__(256) em_xtiles_kernel(const uint32_t *__restrict__ packed,
                                                        int64_t nwords,
                                                        const XSeq *__restrict__ seqs, int kp,
                                                        int nt, uint8_t *__restrict__ xt) {
    const XSeq sq = seqs[blockIdx.x];
    const int j = threadIdx.x % nt, part = threadIdx.x / nt, nparts = 256 / nt;
    const int chunks = kp / 8;
    const size_t xbytes = (size_t)nt * kp * 2;
    const int ntiles = (sq.ns + nt - 1) / nt;
    for (int tt = 0; tt < ntiles; ++tt) {
        uint8_t *dst = xt + (size_t)(sq.tile + tt) * xbytes;
        const int r = tt * nt + j;
        const bool row_ok = r < sq.ns;
        const uint64_t win = row_ok ? window64(packed, nwords, sq.base + r) : 0ull;
        for (int kb = part; kb < chunks; kb += nparts) {
            uint32_t w0 = 0u, w1 = 0u, w2 = 0u, w3 = 0u;
            const int p0 = 2 * kb, p1 = 2 * kb + 1;
            if (row_ok && p0 < sq.l) {
                const uint32_t code = (uint32_t)(win >> (2 * p0)) & 3u;
                const uint32_t v = 0x3F80u << (16 * (code & 1u));
                if (code >> 1) w1 = v; else w0 = v;
            }
            if (row_ok && p1 < sq.l) {
                const uint32_t code = (uint32_t)(win >> (2 * p1)) & 3u;
                const uint32_t v = 0x3F80u << (16 * (code & 1u));
                if (code >> 1) w3 = v; else w2 = v;
            }
            *reinterpret_cast<uint4 *>(dst + tc::kmajor_off(j, 8 * kb, kp)) = make_uint4(w0, w1, w2, w3);
        }
    }
}

// 2^(v - m) for the nv valid entries of a half tile, 0 elsewhere; returns
// their sum (tree order).  The subtractions and the sum use the packed
// two-wide FP32 adds (each lane rounded as a scalar add).
__device__ __forceinline__ float exp_half(float (&v)[32], float m, int nv) {
    const float2 mm = make_float2(-m, -m);
#pragma unroll
    for (int q = 0; q < 32; q += 2) {
        const float2 d = __fadd2_rn(make_float2(v[q], v[q + 1]), mm);
        v[q] = ex2(d.x);
        v[q + 1] = ex2(d.y);
    }
    if (nv < 32) {
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] = q < nv ? v[q] : 0.f;
    }
    float2 part[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
        part[q] = __fadd2_rn(make_float2(v[2 * q], v[2 * q + 1]),
                             make_float2(v[2 * q + 16], v[2 * q + 17]));
#pragma unroll
    for (int w = 4; w >= 1; w >>= 1)
#pragma unroll
        for (int q = 0; q < w; ++q) part[q] = __fadd2_rn(part[q], part[q + w]);
    return part[0].x + part[0].y;
}

__device__ __forceinline__ float max_half(const float (&v)[32], int nv) {
    float mx[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) mx[q] = -INFINITY;
#pragma unroll
    for (int q = 0; q < 32; ++q)
        if (q < nv) mx[q & 7] = fmaxf(mx[q & 7], v[q]);
#pragma unroll
    for (int q = 1; q < 8; ++q) mx[0] = fmaxf(mx[0], mx[q]);
    return mx[0];
}

// The CTA has 128 H + 32 threads (H = 2: 288, two CTAs per SM; H = 4: 544, one
// CTA per SM).  Warps 0 .. 4H-1 compute the softmax: warps w, w + 4, ... share
// the tensor-memory lanes 32*(w%4) .. +31 (candidate rows), warp w taking
// l-mers 32*(w/4) .. +31 of each tile; the H threads of a row share one
// reference maximum m, keep their own compensated sums (added together through
// shared memory at a sequence end), and each reads and accumulates the 8-column
// chunks h, h + H, ... of the row's count columns.  Warp 4H issues the MMAs
// (the warp runs converged and one lane chosen by elect.sync issues each MMA
// and commit), so issuing never stalls the softmax warps.
//
// Pipeline over the tiles j = 0 .. n-1 of an item, linked by mbarriers:
//   issuer: S(0), S(1); then per j: [P(j) written] O (+)= P X(j);
//           [X(j+2) landed, (E-step only) S buffer of j read] S(j+2) = W X(j+2)^T
//   softmax, per j: [S(j) ready] read S(j), (E-step only) release its buffer;
//           P = 2^(S-m); write P(j) over S(j); [count MMA of j-1 done] read the
//           O of a sequence that ended with tile j-1, announce P(j); one thread
//           starts the copy of X(j+3) into the slot of tile j-1.
// Two score buffers in tensor memory (each holding S(j), then P(j)) and a ring
// of four one-hot tiles in shared memory.  S(j+2) overwrites P(j) only after
// the count MMA that reads P(j): tcgen05.mma operations issued by one thread
// execute in issue order.
//
// Reference maximum: P = 2^(S - m) with m = top - 100, top = sum_p max_a W the
// highest score the row can reach.  When the row's score range sum_p (max_a W
// - min_a W) is <= 200 every score lies in [top - 200, top], so every P is in
// [2^-100, 2^100]: nothing overflows or leaves the normal FP32 (and BF16)
// range.  Rows with a wider range (careful mode, CTA-wide) use the exact
// maximum of each sequence's first tile and the threads of a row compare
// every tile: if a part's sum exceeds 2^64 (or is not finite) m is raised to
// the tile's exact maximum, the row's sums and O are rescaled and the tile
// recomputed.
template <int KP, int H>
__global__ void __launch_bounds__(tc_threads<H>(), (KP <= 80 && H == 2 ? 2 : 1))
    em_tc_kernel(const EmTcParams P) {
    using LY = TcLayout<KP, H>;
    constexpr int NT = LY::NT;
    constexpr int SOFT = soft_threads<H>();
    constexpr int THREADS = tc_threads<H>();
    constexpr int CPT = LY::CPT;  // 8-column count chunks per thread: h, h + H, ...
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbSfull[2], mbSfree[2], mbXfull[LY::NX], mbPfull, mbO, mbEnd;
    __shared__ uint32_t tmem_slot;
    __shared__ float sh_x[2][H][kTcRows];  // [slot][part][row] values shared by a row's H threads
    __shared__ bool s_last;
    __shared__ float s_inv[kTcRows];  // 1 / (sites + 4 pseudocount) per candidate of a fold
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool issuer = warp == SOFT / 32;
    const int quad = warp & 3, half = (warp >> 2) % H;  // half: this thread's part of the row
    const int row = 32 * quad + lane;
    uint8_t *sWhi = smem + LY::OFF_WHI, *sWlo = smem + LY::OFF_WLO, *sX = smem + LY::OFF_X;

    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&mbSfull[b], 1);
            tc::mbar_init(&mbSfree[b], SOFT);
        }
        for (int s = 0; s < LY::NX; ++s) tc::mbar_init(&mbXfull[s], 1);  // + the copy's bytes
        tc::mbar_init(&mbPfull, SOFT);
        tc::mbar_init(&mbO, 1);
        tc::mbar_init(&mbEnd, 1);
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
    const uint32_t tO = tm + 2 * NT;
    const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
    constexpr uint32_t IDESC_S = tc::idesc_bf16(128, NT);
    constexpr uint64_t kXSlot = LY::X_BYTES >> 4;

    // phase trackers (each barrier completes in a fixed order; see above)
    uint32_t phSfull = 0u, phSfree = 0u, phX = 0u, phP = 0u;
    uint32_t o_waited = 0, o_base = 0;  // count MMAs of this CTA known complete / before this item
    uint32_t xcnt = 0;                  // exchanges done (slot = xcnt & 1)
    uint32_t xcopies[LY::NX] = {0u, 0u, 0u, 0u};  // one-hot tile copies issued per slot (thread 0)
    // thread 0: one-hot tile j of the item into ring slot j % NX
    auto copy_x = [&](int64_t tile, int j) {
        const int slot = j % LY::NX;
        tc::mbar_arrive_expect_tx(&mbXfull[slot], (uint32_t)LY::X_BYTES);
        tc::bulk_g2s(sX + slot * LY::X_BYTES, P.xt + tile * LY::X_BYTES, (uint32_t)LY::X_BYTES,
                     &mbXfull[slot]);
        ++xcopies[slot];
    };
    bool ok = true, abort = false;

    auto wait_o = [&](uint32_t target) {  // first `target` count MMAs of the item complete
        while (ok && o_waited < o_base + target) {
            ok = tc::mbar_wait(&mbO, o_waited & 1u, kWaitNs);
            ++o_waited;
        }
    };
    // the sum / maximum over this row's H threads (all of them call it together)
    auto row_reduce = [&](float mine, bool take_max) {
        const int s = xcnt & 1;
        ++xcnt;
        sh_x[s][half][row] = mine;
        tc::named_bar(1 + quad, 32 * H);
        float r = sh_x[s][0][row];
#pragma unroll
        for (int h = 1; h < H; ++h) r = take_max ? fmaxf(r, sh_x[s][h][row]) : r + sh_x[s][h][row];
        return r;
    };

    for (int it = blockIdx.x; it < P.n_items && !abort; it += gridDim.x) {
        const EmItem item = P.items[it];
        const EmInst in = P.inst[item.inst];
        const int l = in.l, L4 = 4 * l;
        const int kq = (L4 + 15) / 16;  // K steps of the score MMA = N / 16 of the count MMA
        const uint32_t idesc_o = tc::idesc_bf16(128, 16 * kq, true);
        const int64_t c = item.c0 + row;
        const bool valid = row < item.nc;
        const int n = item.n_tiles;

        __syncthreads();  // the previous item's MMAs and reads are complete
        if (tid == 0)  // the first NX - 1 one-hot tiles (every slot is free)
            for (int j = 0; j < LY::NX - 1 && j < n; ++j) copy_x(item.tile0 + j, j);
        float span = 0.f;   // sum over this thread's positions of max_a W - min_a W
        float wmax = 0.f;   // sum over this thread's positions of max_a W
        if (!issuer) {
            // W_c = log2 theta_c - log2 bg in FP32, split into BF16 hi + lo: the
            // thread of part h writes the 8-column chunks h, h + H, ... of its row
            float lbg[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) lbg[a] = log2f((float)in.bg[a]);
            for (int k8 = 8 * half; k8 < KP; k8 += 8 * H) {
                float w[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int k = k8 + q;
                    w[q] = (valid && k < L4) ? log2f(__ldcg(P.theta_in + c * P.stride + k)) - lbg[q & 3]
                                             : 0.f;
                }
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const float hi4 = fmaxf(fmaxf(w[4 * g], w[4 * g + 1]), fmaxf(w[4 * g + 2], w[4 * g + 3]));
                    wmax += hi4;
                    span += hi4 - fminf(fminf(w[4 * g], w[4 * g + 1]), fminf(w[4 * g + 2], w[4 * g + 3]));
                }
                uint32_t hi[4], lo[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t h = pack_bf16(w[2 * q], w[2 * q + 1]);
                    hi[q] = h;
                    lo[q] = pack_bf16(w[2 * q] - __uint_as_float(h << 16),
                                      w[2 * q + 1] - __uint_as_float(h & 0xFFFF0000u));
                }
                *reinterpret_cast<uint4 *>(sWhi + tc::kmajor_off(row, k8, KP)) =
                    make_uint4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<uint4 *>(sWlo + tc::kmajor_off(row, k8, KP)) =
                    make_uint4(lo[0], lo[1], lo[2], lo[3]);
            }
        }
        // per row: highest possible score and score range (all parts)
        float row_span = 0.f, row_top = 0.f;
        if (!issuer) {
            row_span = row_reduce(span, false);
            row_top = row_reduce(wmax, false);
        }
        const bool careful = __syncthreads_or(row_span > 200.f);
        if (!issuer) tc::fence_async_smem();
        __syncthreads();  // W is visible to the issuer (the one-hot tiles arrive on mbXfull)

        if (issuer) {
            // The whole warp runs the issue loop: every value an MMA operand or a
            // branch depends on is made warp-uniform (broadcast from lane 0 or
            // voted), so the operands stay in uniform registers, and one elected
            // lane issues each MMA and commit.
            tc::fence_after_sync();
            const uint32_t tmu = __shfl_sync(0xffffffffu, tm, 0);
            const uint32_t tOu = tmu + 2 * NT;
            const int nu = __shfl_sync(0xffffffffu, n, 0);
            const int kqu = __shfl_sync(0xffffffffu, kq, 0);
            const uint32_t idesc_ou = tc::idesc_bf16(128, 16 * kqu, true);
            // operand descriptors; a start address advances by adding (bytes >> 4)
            const uint64_t dWhi = tc::sdesc(tc::smem_addr(sWhi), 128, KP * 16);
            const uint64_t dWlo = tc::sdesc(tc::smem_addr(sWlo), 128, KP * 16);
            const uint64_t dXk = tc::sdesc(tc::smem_addr(sX), 128, KP * 16);   // K-major
            const uint64_t dXmn = tc::sdesc(tc::smem_addr(sX), KP * 16, 128);  // MN-major
            auto issue_scores = [&](uint32_t d, uint32_t slot) {
                const uint64_t dx = dXk + slot * kXSlot;
#pragma unroll
                for (int s = 0; s < KP / 16; ++s)
                    if (s < kqu) tc::mma_bf16_w(d, dWhi + 16 * s, dx + 16 * s, IDESC_S, s > 0);
#pragma unroll
                for (int s = 0; s < KP / 16; ++s)
                    if (s < kqu) tc::mma_bf16_w(d, dWlo + 16 * s, dx + 16 * s, IDESC_S, 1u);
            };
            auto wait_all = [&](uint64_t *bar, uint32_t parity) {
                return __all_sync(0xffffffffu, tc::mbar_wait(bar, parity, kWaitNs) ? 1 : 0) != 0;
            };
            ok = wait_all(&mbXfull[0], phX & 1u);
            phX ^= 1u;
            tc::fence_after_sync();
            issue_scores(tmu, 0);
            tc::mma_commit_w(&mbSfull[0]);
            if (nu > 1 && ok) {
                ok = wait_all(&mbXfull[1], (phX >> 1) & 1u);
                phX ^= 2u;
                tc::fence_after_sync();
                issue_scores(tmu + NT, 1);
                tc::mma_commit_w(&mbSfull[1]);
            }
            TileIt<NT> ti;
            ti.start(in, item.seq_lo, item.seq_hi);
            for (int j = 0; j < nu && ok; ++j) {
                if (P.mstep) {
                    ok = wait_all(&mbPfull, phP);
                    phP ^= 1u;
                    tc::fence_after_sync();
                    const uint64_t dx = dXmn + (uint32_t)(j % LY::NX) * kXSlot;
                    // O restarts with a sequence
                    const uint32_t acc0 = __shfl_sync(0xffffffffu, ti.j0 > 0 ? 1u : 0u, 0);
                    // P(j) in score buffer j&1: l-mers 16s..16s+15 at columns
                    // 32(s/2) + 8(s%2) (hi) and 16 further (lo)
                    const uint32_t tP = tmu + NT * (uint32_t)(j & 1);
#pragma unroll
                    for (int s = 0; s < NT / 16; ++s)
                        tc::mma_bf16_ts_w(tOu, tP + 32 * (s >> 1) + 8 * (s & 1), dx + 2 * KP * s,
                                          idesc_ou, s > 0 ? 1u : acc0);
#pragma unroll
                    for (int s = 0; s < NT / 16; ++s)
                        tc::mma_bf16_ts_w(tOu, tP + 32 * (s >> 1) + 16 + 8 * (s & 1),
                                          dx + 2 * KP * s, idesc_ou, 1u);
                    tc::mma_commit_w(&mbO);
                }
                if (j + 2 < nu && ok) {
                    const uint32_t xs = (uint32_t)((j + 2) % LY::NX), b = (uint32_t)(j & 1);
                    ok = wait_all(&mbXfull[xs], (phX >> xs) & 1u);
                    phX ^= 1u << xs;
                    // an M-step's count MMA j, issued above after P(j) was written
                    // (so after S(j) was read), precedes this MMA: no release needed
                    if (!P.mstep) {
                        if (ok) ok = wait_all(&mbSfree[b], (phSfree >> b) & 1u);
                        phSfree ^= 1u << b;
                    }
                    tc::fence_after_sync();
                    issue_scores(tmu + NT * b, xs);
                    tc::mma_commit_w(&mbSfull[b]);
                }
                ti.advance(in, item.seq_hi);
            }
        } else {
            // this item's normalised counts of candidate c, this thread's chunks:
            // tot[8 r + e] holds column 8 (half + H r) + e
            float tot[8 * CPT];
#pragma unroll
            for (int q = 0; q < 8 * CPT; ++q) tot[q] = 0.f;
            // per-sequence log-likelihoods and (ZOOPS) expected site counts, summed
            // in compensated FP32 (the FP64 pipe is narrow on this part)
            float ll_s = 0.f, ll_c = 0.f, zs_s = 0.f, zs_c = 0.f;
            const bool zoops = in.gamma < 1.0;
            const float log_gamma = zoops ? logf((float)in.gamma) : 0.f;
            const float log_no = zoops ? log1pf(-(float)in.gamma) : 0.f;
            // a finished sequence's O is added to tot (scaled by o_inv) during the
            // next tile, before that tile's count MMA restarts O, so the wait for
            // the sequence's last count MMA overlaps the next tile's softmax
            bool o_pend = false;
            float o_inv = 0.f;
            auto read_o = [&]() {
#pragma unroll
                for (int r = 0; r < CPT; ++r) {
                    const int c8 = 8 * (half + H * r);
                    if (c8 < KP) {
                        float o[8];
                        tc::tmem_ld8(tO + lane_base + c8, o);
#pragma unroll
                        for (int q = 0; q < 8; ++q) tot[8 * r + q] += o[q] * o_inv;
                    }
                }
                o_pend = false;
            };
            o_base = o_waited;  // every count MMA of earlier items was waited for
            const uint32_t tS0 = tm + 32 * half + lane_base;  // this thread's columns of buffer 0

            // The tile loop, compiled once per (M-step, careful) pair so that the
            // common case (M-step, fixed reference maximum) carries no branch of
            // the other three; sequences outside, their tiles inside.
            auto run = [&](auto ms_t, auto cf_t) {
                constexpr bool MS = decltype(ms_t)::value, CF = decltype(cf_t)::value;
                int i = 0;  // tile of the item
                for (int seq = item.seq_lo; seq < item.seq_hi; ++seq) {
                    const int ns = in.seq_off[seq + 1] - in.seq_off[seq] - l + 1;  // starts
                    const int ntl = (ns + NT - 1) / NT;
                    // every score of a row lies in [top - 200, top] unless the CTA
                    // is careful, so P = 2^(S - m) stays within [2^-100, 2^100]
                    float m = CF ? -INFINITY : row_top - 100.f;
                    float Ssum = 0.f, Scmp = 0.f;
                    for (int q = 0; q < ntl; ++q, ++i) {
                        const uint32_t b = (uint32_t)(i & 1);
                        const uint32_t tS = tS0 + NT * b;
                        if (ok) ok = tc::mbar_wait(&mbSfull[b], (phSfull >> b) & 1u, kWaitNs);
                        phSfull ^= 1u << b;
                        tc::fence_after_sync();
                        // valid l-mers of this thread's half (only a last tile is partial)
                        const int nv = q + 1 < ntl ? 32 : max(0, min(32, ns - q * NT - 32 * half));
                        float v[32];
                        tc::tmem_ld32(tS, v);
                        if constexpr (CF) {
                            if (q == 0) m = row_reduce(max_half(v, nv), true);  // exact maximum
                        }
                        const float s0 = Ssum, c0s = Scmp;
                        float add = exp_half(v, m, nv);
                        if constexpr (CF) {
                            const float bigf = !(add <= 18446744073709551616.f) ? 1.f : 0.f;  // 2^64
                            // both warps of the lane group take the same branch (named barriers)
                            if (__any_sync(0xffffffffu, row_reduce(bigf, true) > 0.f)) {
                                // redo the tile with m raised to its exact maximum
                                tc::tmem_ld32(tS, v);
                                const float mh = max_half(v, nv);
                                const float tmax = fmaxf(row_reduce(mh, true), m);
                                const float sc = ex2(m - tmax);
                                Ssum = s0 * sc;
                                Scmp = c0s * sc;
                                m = tmax;
                                if (MS && q > 0) {
                                    wait_o((uint32_t)i);  // O holds every count MMA issued so far
                                    tc::fence_after_sync();
#pragma unroll
                                    for (int r = 0; r < CPT; ++r) {
                                        const int c8 = 8 * (half + H * r);
                                        if (c8 < KP) {
                                            float o[8];
                                            tc::tmem_ld8(tO + lane_base + c8, o);
#pragma unroll
                                            for (int e = 0; e < 8; ++e) o[e] *= sc;
                                            tc::tmem_st8(tO + lane_base + c8, o);
                                        }
                                    }
                                }
                                add = exp_half(v, m, nv);
                            }
                        }
                        kahan(Ssum, Scmp, add);
                        tc::fence_before_sync();
                        if constexpr (!MS) {
                            if (i + 2 < n) tc::mbar_arrive(&mbSfree[b]);  // the issuer may overwrite S(i)
                        } else {
                            // P over this thread's own score columns: hi of its 32 l-mers
                            // in the first 16, lo in the last 16 (the count MMA of tile
                            // i-2, which read the buffer's previous P, completed before S(i))
#pragma unroll
                            for (int g = 0; g < 2; ++g) {
                                uint32_t hi[8], lo[8];
#pragma unroll
                                for (int e = 0; e < 8; ++e) {
                                    const float a0 = v[16 * g + 2 * e], a1 = v[16 * g + 2 * e + 1];
                                    const uint32_t h = pack_bf16(a0, a1);
                                    hi[e] = h;
                                    const float2 r = __fadd2_rn(
                                        make_float2(a0, a1),
                                        make_float2(-__uint_as_float(h << 16),
                                                    -__uint_as_float(h & 0xFFFF0000u)));
                                    lo[e] = pack_bf16(r.x, r.y);
                                }
                                tc::tmem_st8u(tS + 8 * g, hi);
                                tc::tmem_st8u(tS + 16 + 8 * g, lo);
                            }
                            tc::tmem_wait_st();
                            // count MMA i-1 complete (it read X(i-1), whose slot is
                            // rebuilt below) before count MMA i can be issued: the
                            // parity waits on mbO never fall two phases behind
                            wait_o((uint32_t)i);
                            if (o_pend) {  // the previous sequence ended with tile i-1
                                tc::fence_after_sync();
                                read_o();
                            }
                            tc::fence_before_sync();
                            tc::mbar_arrive(&mbPfull);
                        }
                        // one-hot tile of i+3 into the slot of tile i-1 (its MMAs are complete)
                        if (i + LY::NX - 1 < n && tid == 0 && ok)
                            copy_x(item.tile0 + i + LY::NX - 1, i + LY::NX - 1);
                    }
                    // the sequence's log-likelihood term and (M-step) the weight of its counts
                    const float Sf = row_reduce(Ssum - Scmp, false);
                    float w = 1.f;  // posterior probability that the sequence holds a site
                    if (zoops) {
                        // ZOOPS: L_i = log[(1 - gamma) + (gamma / ns) sum_j e^r], in FP32
                        // (FP64 transcendentals are slow here)
                        const float lg = log_gamma - logf((float)ns) + (m + log2f(Sf)) * 0.69314718f;
                        const float hi = fmaxf(log_no, lg), lo = fminf(log_no, lg);
                        const float Li = hi + log1pf(expf(lo - hi));
                        w = expf(lg - Li);
                        kahan(ll_s, ll_c, Li);
                    } else {
                        kahan(ll_s, ll_c, (m + log2f(Sf)) * 0.69314718f - logf((float)ns));
                    }
                    kahan(zs_s, zs_c, w);
                    if constexpr (MS) {
                        o_pend = true;  // read during the next tile or after the loop
                        o_inv = w / Sf;
                    }
                }
            };
            if (P.mstep) {
                if (careful) run(std::true_type{}, std::true_type{});
                else run(std::true_type{}, std::false_type{});
            } else {
                if (careful) run(std::false_type{}, std::true_type{});
                else run(std::false_type{}, std::false_type{});
            }
            if (o_pend) {  // the item's last sequence
                wait_o((uint32_t)n);
                tc::fence_after_sync();
                read_o();
                tc::fence_before_sync();
            }
            const double ll = (double)ll_s - (double)ll_c, zs = (double)zs_s - (double)zs_c;
            if (ok && valid && P.G == 1) {
                // the item covers every sequence: final values directly
                if (half == 0) P.ll_out[c] = ll;
                if (P.mstep) {
                    // FP32 (the counts are FP32 sums; FP64 is a narrow pipe here)
                    const float inv =
                        1.f / (float)((in.gamma < 1.0 ? zs : (double)in.t) + 4.0 * (double)P.beta);
                    float *dst = P.theta_out + c * P.stride;
#pragma unroll
                    for (int r = 0; r < CPT; ++r)
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int col = 8 * (half + H * r) + q;
                            if (col < L4) dst[col] = (tot[8 * r + q] + P.beta) * inv;
                        }
                }
            } else if (ok && valid) {
                if (half == 0) {
                    P.part_ll[(int64_t)item.g * P.C + c] = ll;
                    P.part_zs[(int64_t)item.g * P.C + c] = zs;
                }
                if (P.mstep) {
                    float *dst = P.part_acc + ((int64_t)item.g * P.C + c) * P.stride;
#pragma unroll
                    for (int r = 0; r < CPT; ++r)
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int col = 8 * (half + H * r) + q;
                            if (col < L4) dst[col] = tot[8 * r + q];
                        }
                }
            }
        }
        const bool fold = P.G > 1 && P.G <= kFoldMaxG;
        if (fold) __threadfence();  // this thread's partial results are visible device-wide
        abort = __syncthreads_or(!ok);
        if (abort) break;
        // the last of the tile's G items folds the partial results in group
        // order: theta = (sum_g counts + pseudocount) / (t + 4 pseudocount),
        // LL = sum_g LL_g (larger G: em_tc_reduce_kernel after the launch)
        if (fold) {
            if (tid == 0) s_last = atomicAdd(&P.tile_done[it / P.G], 1u) == (uint32_t)(P.G - 1);
            __syncthreads();
        }
        if (fold && s_last) {
            __threadfence();
            if (P.mstep && tid < item.nc) {
                double sites = (double)in.t;  // OOPS: one site per sequence
                if (in.gamma < 1.0) {
                    sites = 0.0;
                    for (int g = 0; g < P.G; ++g)
                        sites += __ldcg(P.part_zs + (int64_t)g * P.C + item.c0 + tid);
                }
                s_inv[tid] = 1.f / (float)(sites + 4.0 * (double)P.beta);
            }
            __syncthreads();
            const int width = P.mstep ? L4 : 0;
            for (int e = tid; e < item.nc * (width + 1); e += THREADS) {
                const int cc = e / (width + 1), q = e - cc * (width + 1);
                const int64_t cg = item.c0 + cc;
                if (q < width) {
                    float acc = 0.f;
                    for (int g = 0; g < P.G; ++g)
                        acc += __ldcg(P.part_acc + ((int64_t)g * P.C + cg) * P.stride + q);
                    P.theta_out[cg * P.stride + q] = (acc + P.beta) * s_inv[cc];
                } else {
                    double acc = 0.0;
                    for (int g = 0; g < P.G; ++g) acc += __ldcg(P.part_ll + (int64_t)g * P.C + cg);
                    P.ll_out[cg] = acc;
                }
            }
            if (tid == 0) P.tile_done[it / P.G] = 0u;  // ready for the next launch
        }
    }
    if (abort && tid == 0) atomicExch(P.err, 1);
    // every one-hot tile copy this CTA issued has landed (bounded) before it exits
    if (tid == 0)
        for (int s = 0; s < LY::NX; ++s)
            if (xcopies[s] > 0u) tc::mbar_wait(&mbXfull[s], (xcopies[s] - 1u) & 1u, kWaitNs);
    // every MMA this CTA issued has completed (bounded) before its memory is freed
    if (issuer) tc::mma_commit_w(&mbEnd);  // the lane that issued the MMAs
    tc::mbar_wait(&mbEnd, 0u, kWaitNs);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tm, LY::TMEM_COLS);
    }
}

// M-step theta = (sum_g counts + pseudocount) / (t + 4 pseudocount) and the
// log-likelihood sum over the G sequence groups, in group order (used when G
// is above kFoldMaxG).
__global__ void em_tc_reduce_kernel(const float *__restrict__ part_acc,
                                    const double *__restrict__ part_ll,
                                    const double *__restrict__ part_zs, int G, int64_t C,
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
    // group sums in group order, the loads of up to 48 groups in flight at a
    // time (adding the zero that pads the last batch changes no sum)
    auto fold = [&](auto load, auto zero) {
        constexpr int kBatch = 48;
        auto s = zero;
        for (int g0 = 0; g0 < G; g0 += kBatch) {
            decltype(zero) v[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) v[u] = g0 + u < G ? load(g0 + u) : zero;
#pragma unroll
            for (int u = 0; u < kBatch; ++u) s += v[u];
        }
        return s;
    };
    if (mstep && (int)q < 4 * inst[lo].l) {
        const float s = fold([&](int g) { return part_acc[((int64_t)g * C + c) * stride + q]; }, 0.f);
        double sites = (double)inst[lo].t;  // OOPS: one site per sequence
        if (inst[lo].gamma < 1.0) sites = fold([&](int g) { return part_zs[(int64_t)g * C + c]; }, 0.0);
        theta_out[idx] = (s + beta) / (float)(sites + 4.0 * (double)beta);
    }
    if (q == 0) ll_out[c] = fold([&](int g) { return part_ll[(int64_t)g * C + c]; }, 0.0);
}

template <int KP, int H>
int launch_tc(const EmTcParams &P, int grid, cudaStream_t st) {
    using LY = TcLayout<KP, H>;
    PROJ_CUDA_TRY(cudaFuncSetAttribute(em_tc_kernel<KP, H>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, LY::TOTAL));
    {
        TraceSpan ts_("em_tc", st);
        em_tc_kernel<KP, H><<<grid, tc_threads<H>(), LY::TOTAL, st>>>(P);
    }
    PROJ_LAUNCH_CHECK("em_tc_kernel");
    return PROJ_OK;
}

template <int KP, int H>
int ctas_per_sm_kp() {
    using LY = TcLayout<KP, H>;
    const int by_tmem = 512 / (int)LY::TMEM_COLS;
    // shared memory: 228 KB per SM, 1 KB reserved per CTA, plus the static part
    int by_smem = 1, by_regs = 1;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, em_tc_kernel<KP, H>) == cudaSuccess) {
        by_smem = 228 * 1024 / (LY::TOTAL + (int)fa.sharedSizeBytes + 1024);
        // registers are granted per pair of warps
        const int threads = (tc_threads<H>() + 63) / 64 * 64;
        by_regs = 65536 / std::max(1, fa.numRegs * threads);
    } else {
        (void)cudaGetLastError();
    }
    return std::max(1, std::min(std::min(by_smem, by_regs), by_tmem));
}

template <int H>
int ctas_per_sm_h(int kp) {
    switch (kp) {
        case 16: return ctas_per_sm_kp<16, H>();
        case 32: return ctas_per_sm_kp<32, H>();
        case 48: return ctas_per_sm_kp<48, H>();
        case 64: return ctas_per_sm_kp<64, H>();
        case 80: return ctas_per_sm_kp<80, H>();
        case 96: return ctas_per_sm_kp<96, H>();
        case 112: return ctas_per_sm_kp<112, H>();
        default: return ctas_per_sm_kp<128, H>();
    }
}

int ctas_per_sm(int kp, int h) { return h == 4 ? ctas_per_sm_h<4>(kp) : ctas_per_sm_h<2>(kp); }

template <int H>
int dispatch_h(int kp, const EmTcParams &P, int grid, cudaStream_t st) {
    switch (kp) {
        case 16: return launch_tc<16, H>(P, grid, st);
        case 32: return launch_tc<32, H>(P, grid, st);
        case 48: return launch_tc<48, H>(P, grid, st);
        case 64: return launch_tc<64, H>(P, grid, st);
        case 80: return launch_tc<80, H>(P, grid, st);
        case 96: return launch_tc<96, H>(P, grid, st);
        case 112: return launch_tc<112, H>(P, grid, st);
        default: return launch_tc<128, H>(P, grid, st);
    }
}

int dispatch(int kp, int h, const EmTcParams &P, int grid, cudaStream_t st) {
    return h == 4 ? dispatch_h<4>(kp, P, grid, st) : dispatch_h<2>(kp, P, grid, st);
}

}  // namespace

// ---------------------------------------------------------------------------
// Work plan and autotuning.  A schedule is (ctas, waves, h): CTAs per SM of the
// persistent grid (<= what shared memory, registers and tensor memory allow),
// when there are fewer candidate tiles than CTA slots how many rounds of the
// slots the sequence-group split fills, and the kernel's parts per row h (2:
// tiles of 64 l-mers, 4: tiles of 128).  The first search of each shape class
// times one M-step launch of every candidate schedule on its own data and keeps
// the fastest (per process); PROJ_AUTOTUNE=0 turns this off (default schedule)
// and PROJ_EM_SCHED="ctas,waves[,h]" forces one.
// ---------------------------------------------------------------------------
namespace {

struct Sched { int ctas, waves, h; };
const Sched kScheds[] = {{2, 1, 2}, {2, 2, 2}, {2, 3, 2}, {2, 4, 2},
                         {1, 1, 4}, {1, 2, 4}, {1, 3, 4}};
constexpr Sched kDefaultSched = {2, 1, 2};

std::mutex g_tune_mu;
std::map<uint64_t, Sched> g_tuned;

uint64_t shape_key(int kp, int64_t C, int tmin, int64_t lmers) {
    int cb = 0, xb = 0;
    while (((int64_t)1 << cb) < C) ++cb;
    while (((int64_t)1 << xb) < lmers) ++xb;
    return ((uint64_t)kp << 48) | ((uint64_t)cb << 40) | ((uint64_t)std::min(tmin, 65535) << 16) |
           (uint64_t)xb;
}

// the one-hot tiles (nt rows each) of every sequence of the run
int build_xtiles(const uint32_t *packed, int64_t nwords, const std::vector<EmInstHost> &insts,
                 int kp, int nt, DevBuf &xt, DevBuf &xseq, cudaStream_t st) {
    std::vector<XSeq> xs;
    int64_t nx = 0;
    for (const EmInstHost &h : insts)
        for (int q = 0; q < h.t; ++q) {
            XSeq v;
            v.base = h.seq_off[q];
            v.tile = nx;
            v.ns = h.seq_off[q + 1] - h.seq_off[q] - h.l + 1;
            v.l = h.l;
            xs.push_back(v);
            nx += (v.ns + nt - 1) / nt;
        }
    const size_t xbytes = (size_t)nt * kp * 2;
    PROJ_TRY(xt.alloc(std::max<int64_t>(1, nx) * xbytes, st));
    PROJ_TRY(xseq.alloc(xs.size() * sizeof(XSeq), st));
    PROJ_CUDA_TRY(cudaMemcpyAsync(xseq.as<XSeq>(), xs.data(), xs.size() * sizeof(XSeq),
                                  cudaMemcpyHostToDevice, st));
    {
        TraceSpan ts_("em_xtiles", st);
        em_xtiles_kernel<<<(unsigned)xs.size(), 256, 0, st>>>(packed, nwords, xseq.as<XSeq>(), kp, nt,
                                                              xt.as<uint8_t>());
    }
    PROJ_LAUNCH_CHECK("em_xtiles_kernel");
    return PROJ_OK;
}

}  // namespace

int em_tc_plan(const std::vector<EmInstHost> &insts, std::vector<EmItem> &items, int &G,
               int ctas, int waves, int h) {
    // split each instance's candidates into tiles of 128; when there are fewer
    // tiles than CTA slots, split the sequences into G groups so that the items
    // fill `waves` rounds of the slots without a partial round
    const int nt = kNT * h / 2;
    int kp = 16;
    int64_t tiles = 0;
    for (const EmInstHost &hi : insts) {
        kp = std::max(kp, 16 * ((4 * hi.l + 15) / 16));
        tiles += (hi.C + kTcRows - 1) / kTcRows;
    }
    const int64_t slots = (int64_t)sm_count() * std::min(ctas, ctas_per_sm(kp, h));
    int tmin = 1 << 30;
    for (const EmInstHost &hi : insts) tmin = std::min(tmin, hi.t);
    G = 1;
    if (tiles > 0 && tiles < slots)
        G = (int)std::min<int64_t>(std::max(1, tmin), std::max<int64_t>(1, waves * slots / tiles));
    items.clear();
    int64_t tb = 0;  // one-hot tiles of the earlier instances
    for (size_t ii = 0; ii < insts.size(); ++ii) {
        const EmInstHost &hi = insts[ii];
        std::vector<int64_t> pre(hi.t + 1, 0);  // tiles of the instance's first q sequences
        for (int q = 0; q < hi.t; ++q)
            pre[q + 1] = pre[q] + (hi.seq_off[q + 1] - hi.seq_off[q] - hi.l + 1 + nt - 1) / nt;
        for (int64_t c0 = 0; c0 < hi.C; c0 += kTcRows)
            for (int g = 0; g < G; ++g) {
                EmItem it;
                it.c0 = hi.cand_begin + c0;
                it.nc = (int)std::min<int64_t>(kTcRows, hi.C - c0);
                it.inst = (int)ii;
                it.seq_lo = (int)((int64_t)hi.t * g / G);
                it.seq_hi = (int)((int64_t)hi.t * (g + 1) / G);
                it.g = g;
                it.n_tiles = (int)(pre[it.seq_hi] - pre[it.seq_lo]);
                it.tile0 = tb + pre[it.seq_lo];
                items.push_back(it);
            }
        tb += pre[hi.t];
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
    // PROJ_EM_SCHED="ctas,waves[,h]" forces one schedule (no tuning, no cache)
    if (const char *fs = getenv("PROJ_EM_SCHED")) {
        int c = 0, g = 0, h = 2;
        const int nf = sscanf(fs, "%d,%d,%d", &c, &g, &h);
        if (nf >= 2 && c >= 1 && c <= 3 && g >= 1 && g <= 8 && (h == 2 || h == 4)) {
            sched = {c, g, h};
            tune = false;
        }
    }

    // buffers sized for the largest G any candidate schedule may pick
    int Gmax = 1;
    std::vector<EmItem> items;
    for (const Sched &sc : kScheds) {
        int G = 1;
        em_tc_plan(insts, items, G, sc.ctas, sc.waves, sc.h);
        Gmax = std::max(Gmax, G);
    }
    {
        int G = 1;
        em_tc_plan(insts, items, G, sched.ctas, sched.waves, sched.h);
        Gmax = std::max(Gmax, G);
    }
    // part_ll, part_zs [G][C] double, then part_acc [G][C][stride] float
    PROJ_TRY(run.part.alloc((size_t)Gmax * C * (2 * sizeof(double) + stride * sizeof(float)), st));
    PROJ_TRY(run.tmp.alloc((size_t)C * stride * sizeof(float), st));
    PROJ_TRY(run.flag.alloc(sizeof(int), st));
    PROJ_CUDA_TRY(cudaMemsetAsync(run.flag.as<int>(), 0, sizeof(int), st));
    int64_t n_tiles = 0;  // candidate tiles (the same for every schedule)
    for (const EmInstHost &h : insts) n_tiles += (h.C + kTcRows - 1) / kTcRows;
    PROJ_TRY(run.tiles.alloc((size_t)std::max<int64_t>(1, n_tiles) * sizeof(uint32_t), st));
    PROJ_CUDA_TRY(cudaMemsetAsync(run.tiles.as<uint32_t>(), 0,
                                  (size_t)std::max<int64_t>(1, n_tiles) * sizeof(uint32_t), st));

    if (tune) {
        // time one M-step launch per schedule on this data (the model copy it
        // updates in place is restored before the real iterations); the one-hot
        // tiles are built once per tile height
        PROJ_CUDA_TRY(cudaMemcpyAsync(run.tmp.as<float>(), theta0, (size_t)C * stride * sizeof(float),
                                      cudaMemcpyDeviceToDevice, st));
        DevBuf ll_scratch, xt2, xs2, xt4, xs4;
        PROJ_TRY(ll_scratch.alloc((size_t)C * sizeof(double), st));
        PROJ_TRY(build_xtiles(packed, nwords, insts, kp, kNT, xt2, xs2, st));
        PROJ_TRY(build_xtiles(packed, nwords, insts, kp, 2 * kNT, xt4, xs4, st));
        cudaEvent_t e0, e1;
        PROJ_CUDA_TRY(cudaEventCreate(&e0));
        PROJ_CUDA_TRY(cudaEventCreate(&e1));
        float best_ms = 1e30f;
        for (const Sched &sc : kScheds) {
            int G = 1;
            const int kpp = em_tc_plan(insts, items, G, sc.ctas, sc.waves, sc.h);
            DevBuf ib;
            PROJ_TRY(ib.alloc(items.size() * sizeof(EmItem), st));
            PROJ_CUDA_TRY(cudaMemcpyAsync(ib.as<EmItem>(), items.data(), items.size() * sizeof(EmItem),
                                          cudaMemcpyHostToDevice, st));
            EmTcParams P{};
            P.packed = packed; P.nwords = nwords; P.inst = inst_dev; P.items = ib.as<EmItem>();
            P.n_items = (int)items.size(); P.theta_in = run.tmp.as<float>(); P.stride = stride;
            P.part_ll = run.part.as<double>(); P.part_zs = run.part.as<double>() + (size_t)G * C;
            P.part_acc = reinterpret_cast<float *>(run.part.as<double>() + (size_t)2 * G * C);
            P.C = C; P.err = run.flag.as<int>(); P.mstep = 1; P.G = G; P.beta = 0.25f;
            P.theta_out = run.tmp.as<float>(); P.ll_out = ll_scratch.as<double>();
            P.tile_done = run.tiles.as<uint32_t>();
            P.xt = (sc.h == 4 ? xt4 : xt2).as<uint8_t>();
            const int grid = (int)std::min<int64_t>(
                (int64_t)items.size(), (int64_t)sm_count() * std::min(sc.ctas, ctas_per_sm(kpp, sc.h)));
            PROJ_CUDA_TRY(cudaEventRecord(e0, st));
            PROJ_TRY(dispatch(kpp, sc.h, P, grid, st));
            if (G > kFoldMaxG) {  // the separate fold is part of this schedule's cost
                const int64_t nq = C * stride;
                em_tc_reduce_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(
                    P.part_acc, P.part_ll, P.part_zs, G, C, stride, inst_dev, (int)insts.size(),
                    P.beta, 1,
                    run.tmp.as<float>(), ll_scratch.as<double>());
                PROJ_LAUNCH_CHECK("em_tc_reduce_kernel");
            }
            PROJ_CUDA_TRY(cudaEventRecord(e1, st));
            PROJ_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            PROJ_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < 0.97f * best_ms) { best_ms = ms; sched = sc; }  // earlier wins near-ties
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = sched;
    }
    run.kp = em_tc_plan(insts, items, run.G, sched.ctas, sched.waves, sched.h);
    run.ctas = sched.ctas;
    run.h = sched.h;
    // the one-hot tiles of every sequence for the chosen tile height, built once
    // for all iterations
    PROJ_TRY(build_xtiles(packed, nwords, insts, kp, kNT * run.h / 2, run.xt, run.xseq, st));
    if (const char *dbg = getenv("PROJ_DEBUG"))
        if (dbg[0] == '1')
            fprintf(stderr, "[projection] em_tc schedule: KP=%d ctas=%d (fit %d) waves=%d h=%d G=%d "
                            "items=%zu tuned=%d\n",
                    run.kp, sched.ctas, ctas_per_sm(run.kp, run.h), sched.waves, run.h, run.G,
                    items.size(), (int)tune);
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
    P.part_zs = run.part.as<double>() + (size_t)G * C;
    P.part_acc = reinterpret_cast<float *>(run.part.as<double>() + (size_t)2 * G * C);
    P.C = C;
    P.G = G;
    P.beta = beta;
    P.theta_out = run.tmp.as<float>();  // in place
    P.ll_out = ll;
    P.tile_done = run.tiles.as<uint32_t>();
    P.xt = run.xt.as<uint8_t>();
    P.err = run.flag.as<int>();
    const int grid = (int)std::min<int64_t>(
        (int64_t)run.n_items, (int64_t)sm_count() * std::min(run.ctas, ctas_per_sm(run.kp, run.h)));
    for (int it = 0; it <= iters; ++it) {
        P.mstep = it < iters;
        PROJ_TRY(dispatch(run.kp, run.h, P, grid, st));
        if (G > kFoldMaxG) {
            const int64_t n = P.mstep ? C * stride : C;
            {
                TraceSpan ts_("em_reduce", st);
                em_tc_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                    P.part_acc, P.part_ll, P.part_zs, G, C, stride, run.inst_dev, run.n_inst, beta,
                    P.mstep,
                    run.tmp.as<float>(), ll);
            }
            PROJ_LAUNCH_CHECK("em_tc_reduce_kernel");
        }
    }
    PROJ_CUDA_TRY(cudaMemcpyAsync(theta_out, run.tmp.as<float>(), (size_t)C * stride * sizeof(float),
                                  cudaMemcpyDeviceToDevice, st));
    return PROJ_OK;
}

int em_tc_finish(EmTcRun &run, cudaStream_t st, int *err_dev) {
    if (run.C == 0) return PROJ_OK;
    if (err_dev) {
        PROJ_CUDA_TRY(cudaMemcpyAsync(err_dev, run.flag.as<int>(), sizeof(int),
                                      cudaMemcpyDeviceToDevice, st));
        return PROJ_OK;
    }
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
                    float beta, float *theta_out, double *ll, cudaStream_t st, int *err_dev) {
    EmTcRun run;
    if (C == 0) return PROJ_OK;
    PROJ_TRY(em_tc_prepare(packed, nwords, insts, inst_dev, theta0, C, stride, run, st));
    PROJ_TRY(run_as_graph(kGraphEm, st, [&](cudaStream_t cs) {
        return em_tc_enqueue(run, iters, beta, theta_out, ll, cs);
    }));
    return em_tc_finish(run, st, err_dev);
}

int run_em_tc(const uint32_t *packed, const Layout &L, const double *bg, const float *theta0,
              int64_t C, int iters, float beta, float *theta_out, double *ll, cudaStream_t st,
              double gamma, int *err_dev) {
    std::vector<EmInstHost> insts(1);
    insts[0].t = L.t;
    insts[0].l = L.l;
    insts[0].C = C;
    insts[0].cand_begin = 0;
    insts[0].lmers = L.x;
    insts[0].seq_off = L.seq_off.data();
    EmInst in{};
    in.seq_off = L.seq_off_dev();
    in.t = L.t;
    in.l = L.l;
    in.bg = bg;
    in.cand_begin = 0;
    in.gamma = gamma;
    DevBuf ib;
    PROJ_TRY(ib.alloc(sizeof(EmInst), st));
    PROJ_CUDA_TRY(cudaMemcpyAsync(ib.as<EmInst>(), &in, sizeof(EmInst), cudaMemcpyHostToDevice, st));
    return run_em_tc_batch(packed, L.nwords, insts, ib.as<EmInst>(), theta0, C, 4 * L.l, iters,
                           beta, theta_out, ll, st, err_dev);
}

}  // namespace proj

// ---------------------------------------------------------------------------
// projection_ex2_peak: the exp2 rate (MUFU ex2.approx) the EM kernel's one
// exponential per score is measured against.  Every thread runs eight
// independent chains x <- 2^-x (values stay in [0.5, 1]).
// ---------------------------------------------------------------------------
namespace proj {
namespace {

__global__ void __launch_bounds__(512) ex2_peak_kernel(int iters, float *sink) {
    float x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = 0.125f * (float)q + 1e-3f * (float)(threadIdx.x & 7);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = ex2(-x[q]);
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc += x[q];
    if (acc == 12345.f) sink[blockIdx.x] = acc;  // keeps the work; never true
}

}  // namespace
}  // namespace proj

extern "C" int projection_ex2_peak(double *ex2_per_s, void *stream) {
    using namespace proj;
    clear_error();
    PROJ_REQUIRE(ex2_per_s != nullptr, "ex2_per_s must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = sm_count() * 4, threads = 512, iters = 4096;
    DevBuf sink;
    PROJ_TRY(sink.alloc((size_t)grid * 4, st));
    cudaEvent_t e0, e1;
    PROJ_CUDA_TRY(cudaEventCreate(&e0));
    PROJ_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {  // first launch warms up; keep the fastest
        PROJ_CUDA_TRY(cudaEventRecord(e0, st));
        ex2_peak_kernel<<<grid, threads, 0, st>>>(iters, sink.as<float>());
        PROJ_CUDA_TRY(cudaEventRecord(e1, st));
        PROJ_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        PROJ_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    PROJ_LAUNCH_CHECK("ex2_peak_kernel");
    *ex2_per_s = (double)grid * threads * iters * 8 / (best * 1e-3);
    return PROJ_OK;
}

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
