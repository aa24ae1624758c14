// Steps a2-a5: random projection h_k, base-4 hashing and bucket counting
// (Algorithm 2 steps 2a-2c; Section 6's base-|Sigma| conversion, A:0 C:1 T:2
// G:3, first projected position most significant), and the enriched buckets
// of Algorithm 2 step 3 (a bucket is enriched when it holds >= s l-mers).
//
// Design (GB300): all trials run in one launch, one 1024-thread CTA per
// (trial, key-range part).  The packed input (2 bits per base) and the
// sequence offsets are staged in shared memory with vectorised loads; each
// thread builds the keys of its l-mers from a 64-bit window of packed codes
// and increments a shared-memory histogram (u32 counters, or u16 pairs when
// 4^k counters of 4 bytes do not fit and no bucket can exceed 65535).  When
// 4^k counters do not fit in one CTA the key space is split into parts, each
// CTA counting only keys in its range.
//
// Two passes give exact, deterministic output without atomics deciding any
// order: pass 1 counts enriched buckets and members per (trial, part); a scan
// gives every (trial, part) its output offsets; pass 2 recounts, writes the
// candidate table in key order, compacts the enriched l-mers in l-mer-id order
// (block-wide ballot scan), and places each one at its bucket's cursor with a
// single warp walking that list (match_any ranks equal keys within a step), so
// members come out ascending within every bucket.
#include <stdlib.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace proj {
namespace {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int kHistBytes = 128 * 1024;    // shared-memory histogram budget
constexpr int kSmemLimit = 226 * 1024;    // dynamic shared memory per CTA (227 KB opt-in
                                          // minus room for the static arrays)
constexpr int kSortChunk = 8192;          // l-mers per (trial, chunk) of the partition
constexpr int kMaxSortChunks = 8192;      // chunks per trial in partitioned mode

struct HashParams {
    const uint32_t *packed;
    int64_t nwords;
    const int32_t *seq_off;   // [t+1]
    const int32_t *lmer_off;  // [t+1]
    int t, l, k, s, x;
    uint64_t seed;
    int64_t trial_begin;
    int parts;                // CTAs per trial
    int hb;                   // buckets per part
    int hist16;               // u16 counters
    int count16;              // partitioned counting pass in 64 KB (see hash_unit)
    int stage_words;          // packed words staged in smem (0 = read global)
    int fixed_pos;            // positions given by the caller
    int pos_in[16];
    const uint8_t *pos_tab;   // [n_trials][k] positions drawn once for the call, or null
                              // (each CTA draws its trial's positions)
    uint8_t *pos_out;
    uint32_t *counts_out;
    // pass 1 outputs
    int32_t *part_nb, *part_nm;
    // pass 2 inputs/outputs
    const int64_t *cand_base, *mem_base;
    int64_t cap_cand, cap_members;
    int32_t *cand_trial;
    uint32_t *cand_key;
    int32_t *cand_cnt;
    int64_t *cand_off;
    int32_t *members;
    uint32_t *scratch_key;    // [cap_members]
    int32_t *scratch_gid;     // [cap_members]
    // partitioned mode (large inputs split into many key-range parts; always u32
    // counters, so key - part * hb < 32768 fits 16 bits): the l-mers of chunk c
    // (ids c*kSortChunk ..) of a trial sit in region (trial*n_chunks + c)*kSortChunk
    // of prel (key - part * hb) and plid (id - c*kSortChunk), grouped by part in
    // l-mer order; part p occupies [pstart[q*(parts+1) + p], pstart[q*(parts+1) + p+1])
    // of region q.  A unit (trial, part) walks its pieces chunk by chunk, i.e. in
    // l-mer order (two 16-bit arrays: the counting pass reads 2 bytes per l-mer).
    int partitioned;
    const uint16_t *prel;
    const uint16_t *plid;
    const int32_t *pstart;
    int n_chunks;
    const int *chunk_info;    // [n_chunks][8]: see chunk_info_kernel
    // counting pass: each unit's enriched buckets as (key - part * hb, size), in
    // key order, at emit[emit_off[unit] ..] (capacity: every enriched bucket
    // holds >= s of the unit's l-mers)
    uint2 *emit;
    const int64_t *emit_off;
};

struct SmemLayout {
    int hist_bytes, bitmap_bytes, cb_bytes, off_bytes, words_bytes, total;
};

// histogram | enriched bitmap (fill) | partitioned: the unit's chunk walk
// (int32 prefix [n_chunks+1], int64 bases [n_chunks]) | else: sequence and
// l-mer offsets, staged packed words
__host__ __device__ inline SmemLayout smem_layout(const HashParams &P, bool fill) {
    SmemLayout S;
    S.hist_bytes = (P.hist16 || (!fill && P.count16) ? 2 : 4) * P.hb;
    S.hist_bytes = (S.hist_bytes + 15) & ~15;
    // enriched-bucket bitmap: the fill pass's, and the u32 counting pass's
    S.bitmap_bytes = (fill || !P.hist16) ? (((P.hb + 31) / 32) * 4 + 15) & ~15 : 0;
    S.cb_bytes = P.partitioned ? (((P.n_chunks + 1) * 4 + 15) & ~15) + P.n_chunks * 8 : 0;
    S.off_bytes = P.partitioned ? 0 : ((2 * (P.t + 1) * 4) + 15) & ~15;
    S.words_bytes = P.stage_words ? ((P.stage_words + 2) * 4 + 15) & ~15 : 0;
    S.total = S.hist_bytes + S.bitmap_bytes + S.cb_bytes + S.off_bytes + S.words_bytes;
    return S;
}


__device__ __forceinline__ uint32_t lmer_key(uint64_t win, const int *pos, int k) {
    uint32_t key = 0u;
#pragma unroll
    for (int q = 0; q < 16; ++q)
        if (q < k) key = (key << 2) | (uint32_t)((win >> (2 * pos[q])) & 3u);
    return key;
}

// The same with the number of projected positions fixed at compile time (K > 0);
// K = 0 falls back to the run-time k.
template <int K>
__device__ __forceinline__ uint32_t lmer_key_k(uint64_t win, const int *pos, int k) {
    if constexpr (K == 0) {
        return lmer_key(win, pos, k);
    } else {
        uint32_t key = 0u;
#pragma unroll
        for (int q = 0; q < K; ++q) key = (key << 2) | (uint32_t)((win >> (2 * pos[q])) & 3u);
        return key;
    }
}

// Block-wide exclusive scan of two ints; returns the prefixes and the totals.
template <int NT = kThreads>
__device__ inline void block_scan2(int a, int b, int &pa, int &pb, int &ta, int &tb,
                                   int2 *warp_tot) {
    constexpr int kWarps = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int va = __shfl_up_sync(0xffffffffu, ia, o);
        const int vb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) { ia += va; ib += vb; }
    }
    if (lane == 31) warp_tot[warp] = make_int2(ia, ib);
    __syncthreads();
    if (warp == 0) {
        int2 v = lane < kWarps ? warp_tot[lane] : make_int2(0, 0);
        int sa = v.x, sb = v.y;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int va = __shfl_up_sync(0xffffffffu, sa, o);
            const int vb = __shfl_up_sync(0xffffffffu, sb, o);
            if (lane >= o) { sa += va; sb += vb; }
        }
        if (lane < kWarps) warp_tot[lane] = make_int2(sa - v.x, sb - v.y);  // exclusive
        if (lane == kWarps - 1) warp_tot[kWarps] = make_int2(sa, sb);        // totals
    }
    __syncthreads();
    pa = warp_tot[warp].x + ia - a;
    pb = warp_tot[warp].y + ib - b;
    ta = warp_tot[kWarps].x;
    tb = warp_tot[kWarps].y;
    __syncthreads();
}

// Partitioned mode: the pieces of unit (trial, part) in chunk order.  Piece c
// holds the unit's flat entries [cb[c], cb[c+1]), entry f of it at
// prel/plid[pb[c] + f].  Ends with a CTA barrier.
// With n_chunks <= blockDim.x the caller may pass thread i's piece bounds
// (pf.x, pf.y) of chunk i, loaded ahead of time.
template <int NT = kThreads>
__device__ inline void unit_walk_setup(const HashParams &P, int trial_local, int part,
                                       int32_t *cb, long long *pb, int2 *s_warp,
                                       const int2 *pf = nullptr) {
    const int per = (P.n_chunks + (int)blockDim.x - 1) / (int)blockDim.x;
    const int c0 = min((int)threadIdx.x * per, P.n_chunks), c1 = min(c0 + per, P.n_chunks);
    const int32_t *ps = P.pstart + (int64_t)trial_local * P.n_chunks * (P.parts + 1);
    auto bounds = [&](int c) {
        return (pf && per == 1) ? *pf
                                : make_int2(ps[c * (P.parts + 1) + part], ps[c * (P.parts + 1) + part + 1]);
    };
    int sum = 0;
    for (int c = c0; c < c1; ++c) {
        const int2 ab = bounds(c);
        sum += ab.y - ab.x;
    }
    int pre, pz, tot, tz;
    block_scan2<NT>(sum, 0, pre, pz, tot, tz, s_warp);
    for (int c = c0; c < c1; ++c) {
        const int2 ab = bounds(c);
        cb[c] = pre;
        pb[c] = ((long long)trial_local * P.n_chunks + c) * kSortChunk + ab.x - pre;
        pre += ab.y - ab.x;
    }
    if (threadIdx.x == 0) cb[P.n_chunks] = tot;
    __syncthreads();
}

// One (trial, key-range part) unit of the bucket kernels; `unit` indexes the
// per-unit arrays of P (part_nb, part_nm, cand_base, mem_base).
// Projected positions of trial trial_local (Algorithm 2 step 2a) into s_pos;
// the caller synchronises before reading them.  From the call's table when
// there is one, else the caller's fixed positions or a draw by thread 0.
__device__ __forceinline__ void trial_positions(const HashParams &P, int trial_local, int *s_pos) {
    if (P.pos_tab) {
        if ((int)threadIdx.x < P.k)
            s_pos[threadIdx.x] = P.pos_tab[(int64_t)trial_local * P.k + threadIdx.x];
    } else if (threadIdx.x == 0) {
        if (P.fixed_pos) {
            for (int q = 0; q < P.k; ++q) s_pos[q] = P.pos_in[q];
        } else {
            draw_positions(P.seed, (uint64_t)(P.trial_begin + trial_local), P.l, P.k, s_pos);
        }
    }
}

template <bool FILL, int K, int NT = kThreads>
__device__ __forceinline__ void hash_unit(const HashParams &P, const int unit, uint8_t *smem,
                                          int *s_pos, int2 *s_warp, int *s_round) {
    constexpr int kThreads = NT, kWarps = NT / 32;  // this CTA's size

    const SmemLayout S = smem_layout(P, FILL);
    uint32_t *hist32 = reinterpret_cast<uint32_t *>(smem);
    uint16_t *hist16 = reinterpret_cast<uint16_t *>(smem);
    uint32_t *bitmap = reinterpret_cast<uint32_t *>(smem + S.hist_bytes);
    int32_t *s_cb = reinterpret_cast<int32_t *>(smem + S.hist_bytes + S.bitmap_bytes);
    long long *s_pb = reinterpret_cast<long long *>(
        smem + S.hist_bytes + S.bitmap_bytes + (((P.n_chunks + 1) * 4 + 15) & ~15));
    int32_t *s_seq = reinterpret_cast<int32_t *>(smem + S.hist_bytes + S.bitmap_bytes + S.cb_bytes);
    int32_t *s_lmer = s_seq + (P.t + 1);
    uint32_t *s_words = reinterpret_cast<uint32_t *>(smem + S.hist_bytes + S.bitmap_bytes +
                                                     S.cb_bytes + S.off_bytes);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int trial_local = unit / P.parts;
    const int part = unit % P.parts;
    const uint64_t trial = (uint64_t)(P.trial_begin + trial_local);
    const uint32_t lo_key = (uint32_t)part * (uint32_t)P.hb;
    const uint32_t hb = (uint32_t)P.hb;

    // the unit's piece bounds in chunk tid, loaded before the clear so that
    // their latency overlaps it (partitioned mode, one chunk per thread)
    int2 pf = make_int2(0, 0);
    if (P.partitioned && tid < P.n_chunks && P.n_chunks <= kThreads) {
        const int32_t *ps = P.pstart + ((int64_t)trial_local * P.n_chunks + tid) * (P.parts + 1) + part;
        pf = make_int2(ps[0], ps[1]);
    }
    // projection positions of this trial (Algorithm 2 step 2a); partitioned
    // mode reads keys that are already built and needs them only to report
    // them
    if (!P.partitioned || (!FILL && P.pos_out && part == 0)) trial_positions(P, trial_local, s_pos);
    if (!P.partitioned)
        for (int i = tid; i <= P.t; i += kThreads) {
            s_seq[i] = P.seq_off[i];
            s_lmer[i] = P.lmer_off[i];
        }
    const uint32_t *words = P.packed;
    int64_t nwords = P.nwords;
    if (P.stage_words) {
        const int nw = P.stage_words;
        if ((reinterpret_cast<uintptr_t>(P.packed) & 15u) == 0) {
            const uint4 *src = reinterpret_cast<const uint4 *>(P.packed);
            uint4 *dst = reinterpret_cast<uint4 *>(s_words);
            for (int v = tid; v < nw / 4; v += kThreads) dst[v] = __ldg(src + v);
            for (int w = (nw / 4) * 4 + tid; w < nw + 2; w += kThreads)
                s_words[w] = w < nw ? __ldg(P.packed + w) : 0u;
        } else {
            for (int w = tid; w < nw + 2; w += kThreads) s_words[w] = w < nw ? __ldg(P.packed + w) : 0u;
        }
        words = s_words;
        nwords = nw + 2;
    }
    const int hist_words = S.hist_bytes / 4;  // a multiple of 4
    for (int w = tid; w < hist_words / 4; w += kThreads)
        reinterpret_cast<uint4 *>(hist32)[w] = make_uint4(0u, 0u, 0u, 0u);
    if (FILL || !P.hist16)
        for (int w = tid; w < S.bitmap_bytes / 4; w += kThreads) bitmap[w] = 0u;
    __syncthreads();
    if (!FILL && P.pos_out && part == 0 && tid < P.k)
        P.pos_out[(int64_t)trial_local * P.k + tid] = (uint8_t)s_pos[tid];
    if (P.partitioned) unit_walk_setup<NT>(P, trial_local, part, s_cb, s_pb, s_warp, &pf);

    int pos[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) pos[q] = (q < P.k && !P.partitioned) ? s_pos[q] : 0;

    // Algorithm 2 steps 2b-2c: project every l-mer and count its bucket.  With
    // u32 counters the counting pass also marks, in the bitmap, each bucket at
    // the increment that brings it to s l-mers: the enriched buckets.
    auto bump = [&](uint32_t r) {
        if (!FILL) {
            if (atomicAdd(&hist32[r], 1u) == (uint32_t)(P.s - 1)) atomicOr(&bitmap[r >> 5], 1u << (r & 31u));
        } else {
            atomicAdd(&hist32[r], 1u);
        }
    };
    const int n_flat = P.partitioned ? s_cb[P.n_chunks] : 0;  // the unit's l-mers
    // the unit's keys (relative to its part) in any order: warp w takes pieces
    // w, w + W, ... (W warps), the first 256 entries of four pieces at a time,
    // each lane 32 loads in flight ahead of their increments (the pieces stream
    // from HBM), then what long pieces hold beyond that
    auto walk = [&](auto &&f) {
        for (int c0 = warp; c0 < P.n_chunks; c0 += 4 * kWarps) {
            uint32_t r[4][8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = c0 + j * kWarps;
                const int len = c < P.n_chunks ? min(s_cb[c + 1] - s_cb[c], 256) : 0;
                const uint16_t *src = P.prel + (c < P.n_chunks ? s_pb[c] + s_cb[c] : 0);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int e = lane + 32 * q;
                    r[j][q] = e < len ? (uint32_t)__ldg(src + e) : 0xFFFFFFFFu;
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (r[j][q] != 0xFFFFFFFFu) f(r[j][q]);
        }
        for (int c = warp; c < P.n_chunks; c += kWarps) {
            const int len = s_cb[c + 1] - s_cb[c];
            const uint16_t *src = P.prel + (s_pb[c] + s_cb[c]);
            for (int e0 = 256 + lane; e0 < len; e0 += 8 * 32) {
                uint32_t r[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int e = e0 + 32 * q;
                    r[q] = e < len ? (uint32_t)__ldg(src + e) : 0xFFFFFFFFu;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (r[q] != 0xFFFFFFFFu) f(r[q]);
            }
        }
    };
    if constexpr (!FILL) {
        if (P.count16) {
            // Partitioned counting pass in 64 KB of counters, so that several
            // units share an SM: u16 counters over the part's 2^15 keys when the
            // unit holds at most 65,535 l-mers (no counter can overflow), else two
            // rounds of u32 counters over 2^14 keys each, both walking all the
            // unit's l-mers.  A bucket is marked in the bitmap at the increment
            // that brings it to s; the marks, in key order, are the unit's list.
            const bool wide = n_flat > 65535;  // block-uniform
            const int rounds = wide ? 2 : 1;
            const uint32_t span = wide ? hb / 2 : hb;
            int NBt = 0, NMt = 0;
            for (int rd = 0; rd < rounds; ++rd) {
                const uint32_t k0 = (uint32_t)rd * span;
                if (rd > 0) {
                    for (int w = tid; w < hist_words / 4; w += kThreads)
                        reinterpret_cast<uint4 *>(hist32)[w] = make_uint4(0u, 0u, 0u, 0u);
                    for (int w = tid; w < S.bitmap_bytes / 4; w += kThreads) bitmap[w] = 0u;
                    __syncthreads();
                }
                walk([&](uint32_t r) {
                    const uint32_t q = r - k0;
                    if (q >= span) return;
                    uint32_t c;
                    if (wide) {
                        c = atomicAdd(&hist32[q], 1u);
                    } else {
                        const uint32_t sh = 16u * (q & 1u);
                        c = (atomicAdd(&hist32[q >> 1], 1u << sh) >> sh) & 0xFFFFu;
                    }
                    if (c == (uint32_t)(P.s - 1)) atomicOr(&bitmap[q >> 5], 1u << (q & 31u));
                });
                __syncthreads();
                const int nwb = (int)((span + 31) >> 5);
                const int per = (nwb + kThreads - 1) / kThreads;
                const int w0 = min(tid * per, nwb), w1 = min(w0 + per, nwb);
                auto cnt = [&](uint32_t q) { return wide ? hist32[q] : (uint32_t)hist16[q]; };
                if (P.counts_out) {
                    uint32_t *dst = P.counts_out + (((int64_t)trial_local) << (2 * P.k)) + lo_key + k0;
                    for (uint32_t q = tid; q < span; q += kThreads) dst[q] = cnt(q);
                }
                int nb = 0, nm = 0;
                for (int w = w0; w < w1; ++w) {
                    uint32_t bits = bitmap[w];
                    nb += __popc(bits);
                    while (bits) {
                        const uint32_t q = 32u * w + (uint32_t)(__ffs(bits) - 1);
                        bits &= bits - 1u;
                        nm += (int)cnt(q);
                    }
                }
                int rb, rm, NB, NM;
                block_scan2<NT>(nb, nm, rb, rm, NB, NM, s_warp);
                if (P.emit) {
                    uint2 *dst = P.emit + P.emit_off[unit] + NBt;
                    for (int w = w0; w < w1; ++w) {
                        uint32_t bits = bitmap[w];
                        while (bits) {
                            const uint32_t q = 32u * w + (uint32_t)(__ffs(bits) - 1);
                            bits &= bits - 1u;
                            dst[rb++] = make_uint2(k0 + q, cnt(q));
                        }
                    }
                }
                NBt += NB;
                NMt += NM;
                __syncthreads();  // the next round clears what this one read
            }
            if (tid == 0) {
                P.part_nb[unit] = NBt;
                P.part_nm[unit] = NMt;
            }
            return;
        }
    }
    if (P.partitioned) {
        walk(bump);  // u32 counters in this mode
    } else {
        int i = 0;
        for (int gid = tid; gid < P.x; gid += kThreads) {
            while (s_lmer[i + 1] <= gid) ++i;
            const int64_t b0 = (int64_t)s_seq[i] + (gid - s_lmer[i]);
            const uint32_t rel = lmer_key_k<K>(window64(words, nwords, b0), pos, P.k) - lo_key;
            if (rel < hb) {
                if (P.hist16) atomicAdd(&hist32[rel >> 1], 1u << (16 * (rel & 1u)));
                else bump(rel);
            }
        }
    }
    __syncthreads();

    if (!FILL && P.counts_out) {
        uint32_t *dst = P.counts_out + (((int64_t)trial_local) << (2 * P.k)) + lo_key;
        for (uint32_t b = tid; b < hb; b += kThreads) dst[b] = P.hist16 ? hist16[b] : hist32[b];
    }

    // Algorithm 2 step 3: enriched buckets (count >= s) of this key range.
    if (!FILL && !P.hist16) {
        // counting pass, u32 counters: the enriched buckets are the bitmap's
        // bits; thread i takes a run of its words (key order), and block-scanned
        // offsets keep key order in the unit's list
        const int nwb = (P.hb + 31) >> 5;
        const int per = (nwb + kThreads - 1) / kThreads;
        const int w0 = min(tid * per, nwb), w1 = min(w0 + per, nwb);
        int nb = 0, nm = 0;
        for (int w = w0; w < w1; ++w) {
            uint32_t bits = bitmap[w];
            nb += __popc(bits);
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1u;
                nm += (int)hist32[32 * w + b];
            }
        }
        int rb, rm, NB, NM;  // this thread's first enriched bucket; unit totals
        block_scan2<NT>(nb, nm, rb, rm, NB, NM, s_warp);
        if (P.emit) {  // this unit's enriched buckets, in key order
            uint2 *dst = P.emit + P.emit_off[unit];
            for (int w = w0; w < w1; ++w) {
                uint32_t bits = bitmap[w];
                while (bits) {
                    const uint32_t key = 32u * w + (uint32_t)(__ffs(bits) - 1);
                    bits &= bits - 1u;
                    dst[rb++] = make_uint2(key, hist32[key]);
                }
            }
        }
        if (tid == 0) {
            P.part_nb[unit] = NB;
            P.part_nm[unit] = NM;
        }
        return;
    }
    // Otherwise warp w takes buckets [w*span, (w+1)*span) in rows of 32
    // consecutive buckets, lane i reading bucket row + i (consecutive words: no
    // bank conflicts); a row's ballot and lane scan keep key order.
    const int span = (((P.hb + kWarps - 1) / kWarps) + 31) & ~31;
    const int wb = min(warp * span, P.hb), we = min(wb + span, P.hb);
    int nb = 0, nm = 0;
    for (int r = wb; r < we; r += 32) {
        const int b = r + lane;
        const int c = b < we ? (P.hist16 ? (int)hist16[b] : (int)hist32[b]) : 0;
        if (c >= P.s) { ++nb; nm += c; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nb += __shfl_xor_sync(0xffffffffu, nb, o);
        nm += __shfl_xor_sync(0xffffffffu, nm, o);
    }
    int rb, rm, NB, NM;  // this warp's first enriched bucket and member offset; unit totals
    block_scan2<NT>(lane == 0 ? nb : 0, lane == 0 ? nm : 0, rb, rm, NB, NM, s_warp);
    rb = __shfl_sync(0xffffffffu, rb, 0);
    rm = __shfl_sync(0xffffffffu, rm, 0);

    if (!FILL) {
        if (P.emit) {  // this unit's enriched buckets, in key order
            uint2 *dst = P.emit + P.emit_off[unit];
            for (int r = wb; r < we; r += 32) {
                const int b = r + lane;
                const int c = b < we ? (P.hist16 ? (int)hist16[b] : (int)hist32[b]) : 0;
                const bool e = c >= P.s;
                const uint32_t bal = __ballot_sync(0xffffffffu, e);
                if (e) dst[rb + __popc(bal & ((1u << lane) - 1u))] = make_uint2((uint32_t)b, (uint32_t)c);
                rb += __popc(bal);
            }
        }
        if (tid == 0) {
            P.part_nb[unit] = NB;
            P.part_nm[unit] = NM;
        }
        return;
    }

    // pass 2: candidate table in key order, bucket cursors, enriched bitmap
    const int64_t cbase = P.cand_base[unit];
    const int64_t mbase = P.mem_base[unit];
    for (int r = wb; r < we; r += 32) {
        const int b = r + lane;
        const int c = b < we ? (P.hist16 ? (int)hist16[b] : (int)hist32[b]) : 0;
        const bool e = c >= P.s;
        const uint32_t bal = __ballot_sync(0xffffffffu, e);
        int v = e ? c : 0;  // inclusive lane scan of the enriched sizes of this row
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (e) {
            const int64_t ci = cbase + rb + __popc(bal & ((1u << lane) - 1u));
            const int mo = rm + v - c;
            if (ci < P.cap_cand) {
                P.cand_trial[ci] = (int32_t)trial;
                P.cand_key[ci] = lo_key + (uint32_t)b;
                P.cand_cnt[ci] = c;
                P.cand_off[ci] = mbase + mo;
            }
            if (P.hist16) hist16[b] = (uint16_t)mo; else hist32[b] = (uint32_t)mo;
        }
        if (lane == 0) bitmap[b >> 5] = bal;  // rows are 32-aligned: one bitmap word each
        rb += __popc(bal);
        rm += __shfl_sync(0xffffffffu, v, 31);
    }
    __syncthreads();
    if (mbase + NM > P.cap_members || NM == 0) return;  // block-uniform

    // enriched l-mers in id order -> scratch[mbase .. mbase+NM)
    {
        int i = 0, running = 0, c = 0;
        const int64_t n_iter = P.partitioned ? (int64_t)n_flat : (int64_t)P.x;
        for (int64_t base = 0; base < n_iter; base += kThreads) {
            const int64_t it = base + tid;
            bool e = false;
            uint32_t rel = 0u;
            int gid = 0;
            if (it < n_iter) {
                if (P.partitioned) {
                    while (s_cb[c + 1] <= it) ++c;
                    rel = P.prel[s_pb[c] + it];
                    gid = c * kSortChunk + (int)P.plid[s_pb[c] + it];
                } else {
                    gid = (int)it;
                    while (s_lmer[i + 1] <= gid) ++i;
                    const int64_t b0 = (int64_t)s_seq[i] + (gid - s_lmer[i]);
                    rel = lmer_key_k<K>(window64(words, nwords, b0), pos, P.k) - lo_key;
                }
                e = rel < hb && ((bitmap[rel >> 5] >> (rel & 31u)) & 1u);
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, e);
            if (lane == 0) s_round[warp] = __popc(bal);
            __syncthreads();
            if (warp == 0) {
                const int v = lane < kWarps ? s_round[lane] : 0;
                int sc = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, sc, o);
                    if (lane >= o) sc += u;
                }
                if (lane < kWarps) s_round[lane] = sc - v;
                if (lane == kWarps - 1) s_round[kWarps] = sc;
            }
            __syncthreads();
            if (e) {
                const int q = running + s_round[warp] + __popc(bal & ((1u << lane) - 1u));
                P.scratch_key[mbase + q] = rel;
                P.scratch_gid[mbase + q] = gid;
            }
            running += s_round[kWarps];
            __syncthreads();
        }
    }
    __threadfence_block();
    __syncthreads();

    // stable placement at the bucket cursors: the list is taken in rounds of
    // kThreads entries, all loaded at once; the warps then take turns in list
    // order, and within a warp match_any ranks equal keys, so every bucket's
    // members come out ascending
    for (int q0 = 0; q0 < NM; q0 += kThreads) {
        const int q = q0 + tid;
        const bool act = q < NM;
        uint32_t rel = 0u;
        int gid = 0;
        if (act) {
            rel = P.scratch_key[mbase + q];
            gid = P.scratch_gid[mbase + q];
        }
        const unsigned amask = __ballot_sync(0xffffffffu, act);
        unsigned grp = 0u;
        int rank = 0;
        if (act) {
            grp = __match_any_sync(amask, rel);
            rank = __popc(grp & ((1u << lane) - 1u));
        }
        const int nturn = min(kWarps, (NM - q0 + 31) / 32);
        for (int w = 0; w < nturn; ++w) {
            if (warp == w) {
                int cur = 0;
                if (act) cur = P.hist16 ? (int)hist16[rel] : (int)hist32[rel];
                __syncwarp();
                if (act) {
                    P.members[mbase + cur + rank] = gid;
                    if (rank == 0) {
                        const int nxt = cur + __popc(grp);
                        if (P.hist16) hist16[rel] = (uint16_t)nxt; else hist32[rel] = (uint32_t)nxt;
                    }
                }
            }
            __syncthreads();
        }
    }
}

template <bool FILL, int K, int NT>
__global__ void __launch_bounds__(NT, kThreads / NT) hash_kernel(const HashParams P) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_pos[16];
    __shared__ int2 s_warp[NT / 32 + 1];
    __shared__ int s_round[NT / 32 + 1];
    hash_unit<FILL, K, NT>(P, (int)blockIdx.x, smem, s_pos, s_warp, s_round);
}

// Many instances in one launch: block u runs unit u - unit_begin[i] of the
// instance i with unit_begin[i] <= u < unit_begin[i+1].  Each instance's
// parameter block already points at its own slices of the per-unit arrays.
template <bool FILL>
__global__ void __launch_bounds__(kThreads, 1) hash_batch_kernel(const HashParams *__restrict__ insts,
                                                                 const int64_t *__restrict__ unit_begin,
                                                                 int n_inst) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_pos[16];
    __shared__ int2 s_warp[kWarps + 1];
    __shared__ int s_round[kWarps + 1];
    const int64_t u = blockIdx.x;
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (unit_begin[mid] <= u) lo = mid; else hi = mid - 1;
    }
    hash_unit<FILL, 0>(insts[lo], (int)(u - unit_begin[lo]), smem, s_pos, s_warp, s_round);
}

// ---------------------------------------------------------------------------
// Partitioned mode for large inputs: when 4^k counters need several key-range
// parts and x is large, every part's CTA would otherwise rebuild all x keys.
// Instead each (trial, chunk of kSortChunk l-mers) builds its keys once,
// groups them by part inside the CTA (stable, so each group is in l-mer
// order) and writes the groups with a table of where each part starts; the
// bucket kernels of unit (trial, part) then read only their part's piece of
// every chunk.  No step depends on another CTA.
// ---------------------------------------------------------------------------
constexpr int kMaxParts = 32;
constexpr int kPartShift = 15;                  // partitioned mode: u32 counters, 2^15 keys per part
constexpr uint32_t kPartKeys = 1u << kPartShift;
// Nine warps: dense chunks give each warp 32 blocks of 32 bases (so a chunk may
// span up to 288 blocks); other chunks give warps 0-7 1024 l-mers each.
constexpr int kSortWarps = 9;
constexpr int kSortThreads = 32 * kSortWarps;
static_assert((kSortWarps - 1) * 1024 == kSortChunk, "chunk = 8 warps x 1024 l-mers");
// a chunk's packed words and sequence offsets are staged in shared memory
// when they fit (kSortChunk l-mers of length <= 32 always span fewer than
// 2^18 bases, but long runs of short sequences can exceed these)
constexpr int kStageWords = 4096;
constexpr int kStageSeqs = (kSortChunk - kStageWords - 2) / 2 - 1;
// Dense chunks (l-mers spread over at most kDenseBlocks blocks of 32 bases and
// kDenseSeqs sequences, i.e. sequences much longer than l) build their keys 32
// at a time from bit planes into a table indexed by base, one pad word per 32
// keys (conflict-free stores of a lane's 32 consecutive keys).
constexpr int kDenseBlocks = 32 * kSortWarps;
constexpr int kDenseSeqs = 255;
// shared memory: region A (a dense chunk's part masks per block; other chunks
// stage words and offsets there, then the grouped output) | region B (other
// chunks: keys and places by l-mer; a dense chunk: its packed words, then the
// part counts and offsets per block) | region C (a dense chunk's sequence
// offsets) | region D (a dense chunk's grouped output)
constexpr int kRegionA = kDenseBlocks * 33;
constexpr int kDenseCountOff = 1024;  // words of region B before a dense chunk's part counts
constexpr int kSortSmem = (kRegionA + kSortChunk + 2 * (kDenseSeqs + 1) + kSortChunk) * 4;
static_assert(kMaxParts * kDenseBlocks <= kRegionA && 2 * kDenseBlocks + 4 <= kDenseCountOff &&
                  kDenseCountOff + kMaxParts * kDenseBlocks / 2 <= kSortChunk,
              "dense chunk layout: part masks in region A, words and part counts in region B");
static_assert(kRegionA >= kSortChunk && kStageWords + 2 + 2 * (kStageSeqs + 1) <= kRegionA,
              "region A holds the grouped output and the staged input");

// sequence holding global l-mer id g (last i with lmer_off[i] <= g)
__device__ __forceinline__ int seq_of(const int32_t *lmer_off, int t, int g) {
    int lo = 0, hi = t - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(lmer_off + mid) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// bits 0, 2, 4, .. 30 of w moved to bits 0 .. 15
__device__ __forceinline__ uint32_t even_bits(uint32_t w) {
    w &= 0x55555555u;
    w = (w | (w >> 1)) & 0x33333333u;
    w = (w | (w >> 2)) & 0x0F0F0F0Fu;
    w = (w | (w >> 4)) & 0x00FF00FFu;
    return (w | (w >> 8)) & 0x0000FFFFu;
}

// Low (lo) and high (hi) code bits of the 32 bases of packed words w0, w1.
__device__ __forceinline__ void bit_planes(uint32_t w0, uint32_t w1, uint32_t &lo, uint32_t &hi) {
    lo = even_bits(w0) | (even_bits(w1) << 16);
    hi = even_bits(w0 >> 1) | (even_bits(w1 >> 1) << 16);
}

// One level of a 32 x 32 bit-matrix transpose: rows r and r + J (bit J of r
// clear) exchange the block of columns with bit J set in row r for the block
// with it clear in row r + J.  The five levels together map bit c of a[r] to
// bit r of a[c]; they commute.
template <int J, uint32_t M>
__device__ __forceinline__ void transpose_level(uint32_t (&a)[32]) {
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        if ((r & J) == 0) {
            const uint32_t x = ((a[r] >> J) ^ a[r + J]) & M;
            a[r + J] ^= x;
            a[r] ^= x << J;
        }
    }
}

// What every trial's CTA of chunk c needs to know about the chunk, worked out
// once per call: [0] first and [1] last sequence, [2] first packed word,
// [3] words to stage for the l-mer-by-l-mer key build (-1: read global memory),
// [4] dense (bit-plane keys), [5] a dense chunk's last 32-base block.
__global__ void chunk_info_kernel(const HashParams P, int *__restrict__ info) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.n_chunks) return;
    const int g0 = c * kSortChunk, n = min(kSortChunk, P.x - g0);
    const int i0 = seq_of(P.lmer_off, P.t, g0), i1 = seq_of(P.lmer_off, P.t, g0 + n - 1);
    const int64_t b_lo = (int64_t)P.seq_off[i0] + (g0 - P.lmer_off[i0]);
    const int64_t b_last = (int64_t)P.seq_off[i1] + (g0 + n - 1 - P.lmer_off[i1]);
    const int64_t w_lo = b_lo >> 4, w_hi = (b_last + P.l + 15) >> 4;
    const int nst = (w_hi - w_lo <= kStageWords && i1 - i0 + 2 <= kStageSeqs) ? (int)(w_hi - w_lo) + 2
                                                                               : -1;
    // 32-base blocks from base 16 * w_lo (the chunk's first l-mer is in block 0)
    const int64_t vb = (b_last - 16 * w_lo) >> 5;
    int *o = info + 8 * (int64_t)c;
    o[0] = i0;
    o[1] = i1;
    o[2] = (int)w_lo;
    o[3] = nst;
    bool dense = vb < kDenseBlocks && i1 - i0 + 1 <= kDenseSeqs;
    for (int q = i0; dense && q <= i1; ++q) dense = P.seq_off[q + 1] - P.seq_off[q] >= 32;
    o[4] = dense ? 1 : 0;  // (a block of 32 bases then meets at most two sequences)
    o[5] = (int)(vb < kDenseBlocks ? vb : kDenseBlocks);
}

template <int K>
__global__ void __launch_bounds__(kSortThreads, 2) part_sort_kernel(const HashParams P,
                                                                    uint16_t *__restrict__ orel,
                                                                    uint16_t *__restrict__ olid,
                                                                    int32_t *__restrict__ pstart) {
    extern __shared__ __align__(16) uint32_t s_dyn[];
    uint32_t *s_a = s_dyn;                    // region A
    uint32_t *s_key = s_dyn + kRegionA;       // region B: key | place << 20 of chunk l-mer j at [j]
    int32_t *s_doff = reinterpret_cast<int32_t *>(s_key + kSortChunk);  // region C [kDenseSeqs + 1]
    int32_t *s_dlm = s_doff + kDenseSeqs + 1;                             // [kDenseSeqs + 1]
    uint32_t *s_dout = reinterpret_cast<uint32_t *>(s_dlm + kDenseSeqs + 1);  // region D
    __shared__ int s_pos[16];
    __shared__ int s_cnt[kSortWarps][kMaxParts];  // per warp: sizes, then output offsets
    __shared__ int s_tot[kMaxParts + 1];
    const int trial_local = blockIdx.y, chunk = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const unsigned below = (1u << lane) - 1u;
    const int g0 = chunk * kSortChunk;
    const int n = min(kSortChunk, P.x - g0);
    const int *ci = P.chunk_info + 8 * (int64_t)chunk;
    const int i0 = ci[0], i1 = ci[1], w_lo = ci[2], nst = ci[3], vb1 = ci[5];
    const bool dense = K > 0 && ci[4] != 0;
    const bool staged = !dense && nst >= 0;
    uint32_t *s_out = dense ? s_dout : s_a;  // the grouped output
    const int nq = i1 - i0 + 1;  // sequences the chunk touches
    trial_positions(P, trial_local, s_pos);
    // l-mer-by-l-mer key build: words and offsets staged in region A
    uint32_t *s_words = s_a;                                               // [kStageWords + 2]
    int32_t *s_soff = reinterpret_cast<int32_t *>(s_a + kStageWords + 2);  // [kStageSeqs + 1]
    int32_t *s_loff = s_soff + kStageSeqs + 1;
    if (dense) {  // words of blocks 0 .. vb1 + 1 into region B, offsets into region C
        for (int w = tid; w < 2 * vb1 + 4; w += kSortThreads)
            s_key[w] = w_lo + w < P.nwords ? __ldg(P.packed + w_lo + w) : 0u;
        for (int q = tid; q <= nq; q += kSortThreads) {
            s_doff[q] = (int32_t)(P.seq_off[i0 + q] - 16 * (int64_t)w_lo);  // base from 16 * w_lo
            s_dlm[q] = P.lmer_off[i0 + q];
        }
    } else if (staged) {
        for (int w = tid; w < nst; w += kSortThreads)
            s_words[w] = w_lo + w < P.nwords ? __ldg(P.packed + w_lo + w) : 0u;
        for (int q = tid; q <= nq; q += kSortThreads) {
            s_soff[q] = (int32_t)(P.seq_off[i0 + q] - 16 * (int64_t)w_lo);
            s_loff[q] = P.lmer_off[i0 + q];
        }
    }
    __syncthreads();
    int pos[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) pos[q] = q < P.k ? s_pos[q] : 0;

    if constexpr (K > 0) {
        if (dense) {
            // Lane i of warp w takes the 32 bases of block v = 32w + i.  Row
            // 2(K-1-q) of a 32 x 32 bit matrix holds the low code bits of
            // projected position q for the block's 32 starts, row 2(K-1-q)+1 the
            // high bits.  Before the transpose, the rows of the part bits (key
            // bits 15 ..) give by a tree of ANDs the mask of the block's l-mers of
            // every part; transposed, word i is the key of the l-mer starting at
            // base 32v + i, first projected position most significant (Section
            // 6).  An l-mer's place in its part's group is the part's start + the
            // part's l-mers of earlier blocks + those below it in its block's
            // mask: a stable grouping with no ranking rounds.
            uint32_t *s_mask = s_a;  // [kMaxParts][kDenseBlocks]
            uint16_t *s_pc = reinterpret_cast<uint16_t *>(s_key + kDenseCountOff);  // same shape
            const int v = 32 * warp + lane;
            const bool has = v <= vb1;
            uint32_t a[32];
            uint32_t valid = 0u;  // bases of the block where an l-mer of the chunk starts
            int c1 = 0, c2 = 0, split = 32;  // id = base + c1 below split, + c2 from it
            if (has) {
                const int lb0 = 32 * v;
                int q = 0, hi = nq - 1;  // last sequence starting at or before base lb0
                while (q < hi) {
                    const int mid = (q + hi + 1) >> 1;
                    if (s_doff[mid] <= lb0) q = mid; else hi = mid - 1;
                }
                auto starts = [&](int qq, int &cq) {  // sequence qq's bits of the block
                    const int sb = s_doff[qq];
                    cq = s_dlm[qq] - g0 - sb;  // chunk-local id = base + cq
                    const int lo = max(sb, -cq), hi2 = min(sb + (s_dlm[qq + 1] - s_dlm[qq]), n - cq);
                    const int l0 = min(max(lo - lb0, 0), 32), h0 = min(max(hi2 - lb0, 0), 32);
                    const uint32_t mh = h0 >= 32 ? 0xFFFFFFFFu : ((1u << h0) - 1u);
                    const uint32_t ml = l0 >= 32 ? 0xFFFFFFFFu : ((1u << l0) - 1u);
                    return mh & ~ml;
                };
                valid = starts(q, c1);
                if (q + 1 < nq && s_doff[q + 1] < lb0 + 32) {
                    split = s_doff[q + 1] - lb0;
                    valid |= starts(q + 1, c2);
                }
                const uint2 w01 = *reinterpret_cast<const uint2 *>(s_key + 2 * v);
                const uint2 w23 = *reinterpret_cast<const uint2 *>(s_key + 2 * v + 2);
                uint32_t lo0, hi0, lo1, hi1;
                bit_planes(w01.x, w01.y, lo0, hi0);
                bit_planes(w23.x, w23.y, lo1, hi1);
#pragma unroll
                for (int r = 0; r < 32; ++r) a[r] = 0u;
#pragma unroll
                for (int qq = 0; qq < K; ++qq) {
                    a[2 * (K - 1 - qq)] = __funnelshift_r(lo0, lo1, pos[qq]);
                    a[2 * (K - 1 - qq) + 1] = __funnelshift_r(hi0, hi1, pos[qq]);
                }
                // part masks: part bit j is key bit kPartShift + j (zero rows past 2K)
                const uint32_t b0 = a[kPartShift], b1 = a[kPartShift + 1], b2 = a[kPartShift + 2],
                               b3 = a[kPartShift + 3], b4 = a[kPartShift + 4];
                uint32_t t1[2], t2[4], t3[8], t4[16];
                t1[0] = valid & ~b4;
                t1[1] = valid & b4;
#pragma unroll
                for (int u = 0; u < 4; ++u) t2[u] = t1[u >> 1] & ((u & 1) ? b3 : ~b3);
#pragma unroll
                for (int u = 0; u < 8; ++u) t3[u] = t2[u >> 1] & ((u & 1) ? b2 : ~b2);
#pragma unroll
                for (int u = 0; u < 16; ++u) t4[u] = t3[u >> 1] & ((u & 1) ? b1 : ~b1);
#pragma unroll
                for (int u = 0; u < 32; ++u) {
                    const uint32_t mk = t4[u >> 1] & ((u & 1) ? b0 : ~b0);
                    s_mask[u * kDenseBlocks + v] = mk;
                    s_pc[u * kDenseBlocks + v] = (uint16_t)__popc(mk);
                }
                transpose_level<16, 0x0000FFFFu>(a);
                transpose_level<8, 0x00FF00FFu>(a);
                transpose_level<4, 0x0F0F0F0Fu>(a);
                transpose_level<2, 0x33333333u>(a);
                transpose_level<1, 0x55555555u>(a);
            }
            __syncthreads();
            // per part: exclusive prefix of the blocks' counts (nine per lane) and
            // the part's size
            const int nb = vb1 + 1;
            for (int p = warp; p < kMaxParts; p += kSortWarps) {
                uint16_t *row = s_pc + p * kDenseBlocks;
                int c9[9], run = 0;
#pragma unroll
                for (int j = 0; j < 9; ++j) {
                    const int vv = 9 * lane + j;
                    c9[j] = vv < nb ? (int)row[vv] : 0;
                    run += c9[j];
                }
                int sc = run;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, sc, o);
                    if (lane >= o) sc += u;
                }
                int at = sc - run;
#pragma unroll
                for (int j = 0; j < 9; ++j) {
                    const int vv = 9 * lane + j;
                    if (vv < nb) row[vv] = (uint16_t)at;
                    at += c9[j];
                }
                if (lane == 31) s_tot[p] = sc;
            }
            __syncthreads();
            if (warp == 0) {
                const int tv = s_tot[lane];
                int sc = tv;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, sc, o);
                    if (lane >= o) sc += u;
                }
                s_tot[lane] = sc - tv;
                if (lane == 31) s_tot[kMaxParts] = sc;
            }
            __syncthreads();
            if (tid <= P.parts)
                pstart[((int64_t)trial_local * P.n_chunks + chunk) * (P.parts + 1) + tid] = s_tot[tid];
            if (has) {
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    if ((valid >> i) & 1u) {
                        const uint32_t key = a[i], part = key >> kPartShift;
                        const uint32_t mk = s_mask[part * kDenseBlocks + v];
                        const int d = s_tot[part] + (int)s_pc[part * kDenseBlocks + v] +
                                      __popc(mk & ((1u << i) - 1u));
                        const int e = 32 * v + i + (i < split ? c1 : c2);
                        s_dout[d] = (key & (kPartKeys - 1u)) | ((uint32_t)e << 16);
                    }
                }
            }
        }
    }
    if (!dense) {
        // warps 0-7: 1024 l-mers each in rounds of 32 (lane i: l-mer j0 + 32r + i),
        // keys built here.  Five ballots on the part bits give lane p the active
        // lanes of part p, whose running count it keeps; every lane reads both
        // from the lane of its part, so each l-mer's place among its warp's
        // l-mers of its part keeps l-mer order with no shared-memory round trip.
        const int j0 = warp * 1024, j1 = min(j0 + 1024, n);
        int i = 0;  // sequence of this lane's l-mer, relative to i0
        uint32_t run = 0u;  // lane p: this warp's l-mers of part p so far
        for (int r = 0; r < 32; ++r) {
            const int j = j0 + 32 * r + lane;
            const bool act = j < j1;
            const unsigned amask = __ballot_sync(0xffffffffu, act);
            uint32_t key = 0u;
            if (act) {
                const int g = g0 + j;
                if (staged) {  // every word the chunk's l-mers touch is in s_words
                    while (s_loff[i + 1] <= g) ++i;
                    const int b = s_soff[i] + (g - s_loff[i]);
                    const int wi = b >> 4, sh = 2 * (b & 15);
                    const uint64_t lo = (uint64_t)s_words[wi] | ((uint64_t)s_words[wi + 1] << 32);
                    const uint64_t win = sh ? (lo >> sh) | ((uint64_t)s_words[wi + 2] << (64 - sh)) : lo;
                    key = lmer_key_k<K>(win, pos, P.k);
                } else {
                    while (__ldg(P.lmer_off + i0 + i + 1) <= g) ++i;
                    const int64_t b0 = (int64_t)__ldg(P.seq_off + i0 + i) + (g - __ldg(P.lmer_off + i0 + i));
                    key = lmer_key_k<K>(window64(P.packed, P.nwords, b0), pos, P.k);
                }
            }
            const uint32_t part = key >> kPartShift;
            unsigned mine = amask;
#pragma unroll
            for (int bit = 0; bit < 5; ++bit) {
                const unsigned B = __ballot_sync(0xffffffffu, (part >> bit) & 1u);
                mine &= ~(B ^ (0u - ((uint32_t)(lane >> bit) & 1u)));
            }
            const unsigned same = __shfl_sync(0xffffffffu, mine, (int)(part & 31u));
            const uint32_t before = __shfl_sync(0xffffffffu, run, (int)(part & 31u));
            if (act) s_key[j] = key | ((before + __popc(same & below)) << 20);
            run += __popc(mine);
        }
        s_cnt[warp][lane] = (int)run;
        __syncthreads();
        // part p starts at s_tot[p] in the chunk; warp w's entries of part p follow
        // those of warps w' < w
        if (tid < kMaxParts) {
            int a = 0;
            for (int w = 0; w < kSortWarps; ++w) {
                const int v = s_cnt[w][tid];
                s_cnt[w][tid] = a;
                a += v;
            }
            s_tot[tid] = a;
        }
        __syncthreads();
        if (warp == 0) {
            const int v = s_tot[lane];
            int sc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, sc, o);
                if (lane >= o) sc += u;
            }
            s_tot[lane] = sc - v;
            if (lane == 31) s_tot[kMaxParts] = sc;
        }
        __syncthreads();
        if (tid <= P.parts)
            pstart[((int64_t)trial_local * P.n_chunks + chunk) * (P.parts + 1) + tid] = s_tot[tid];
        // stable placement into shared memory: after all of part p of warps
        // w' < w, at the l-mer's place among warp w's l-mers of p; entry =
        // (key - part * hb) | chunk-local id << 16
        for (int j = tid; j < n; j += kSortThreads) {
            const uint32_t v = s_key[j];
            const uint32_t key = v & 0xFFFFFu, part = key >> kPartShift;
            s_out[s_tot[part] + s_cnt[j >> 10][part] + (int)(v >> 20)] =
                (key & (kPartKeys - 1u)) | ((uint32_t)j << 16);
        }
    }
    __syncthreads();
    // the grouped entries, four per thread: keys to orel, ids to olid
    const int64_t region = ((int64_t)trial_local * P.n_chunks + chunk) * kSortChunk;
    const int n4 = n >> 2;
    uint2 *rel4 = reinterpret_cast<uint2 *>(orel + region);
    uint2 *lid4 = reinterpret_cast<uint2 *>(olid + region);
    for (int e4 = tid; e4 < n4; e4 += kSortThreads) {
        const uint4 v = *reinterpret_cast<const uint4 *>(s_out + 4 * e4);
        rel4[e4] = make_uint2(__byte_perm(v.x, v.y, 0x5410), __byte_perm(v.z, v.w, 0x5410));
        lid4[e4] = make_uint2(__byte_perm(v.x, v.y, 0x7632), __byte_perm(v.z, v.w, 0x7632));
    }
    for (int e = 4 * n4 + tid; e < n; e += kSortThreads) {
        const uint32_t v = s_out[e];
        orel[region + e] = (uint16_t)(v & 0xFFFFu);
        olid[region + e] = (uint16_t)(v >> 16);
    }
}

// exclusive scan of n int64 values in one CTA, out[n] = total
__global__ void __launch_bounds__(1024) scan_i64_kernel(const int64_t *__restrict__ in, int64_t n,
                                                        int64_t *__restrict__ out) {
    __shared__ long long s[1024];
    const int tid = threadIdx.x;
    const int64_t chunk = (n + 1023) / 1024;
    const int64_t lo = min((int64_t)tid * chunk, n), hi = min(lo + chunk, n);
    long long a = 0;
    for (int64_t e = lo; e < hi; ++e) a += in[e];
    s[tid] = a;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const long long v = tid >= o ? s[tid - o] : 0;
        __syncthreads();
        s[tid] += v;
        __syncthreads();
    }
    long long p = s[tid] - a;
    for (int64_t e = lo; e < hi; ++e) {
        out[e] = p;
        p += in[e];
    }
    if (tid == 1023) out[n] = s[1023];
}

// Exclusive scan over the (trial, part) counts in launch order, which is
// (trial, key) order: candidate and member offsets plus the totals.
__global__ void __launch_bounds__(1024) hash_scan_kernel(const int32_t *__restrict__ nb,
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
        long long va = tid >= o ? s_a[tid - o] : 0, vb = tid >= o ? s_b[tid - o] : 0;
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

// cand_off[C] = total members (C = totals[0]) when it fits the capacity.
__global__ void cand_end_kernel(const int64_t *__restrict__ totals, int64_t cap_cand,
                                int64_t *__restrict__ cand_off) {
    if (totals[0] <= cap_cand) cand_off[totals[0]] = totals[1];
}

// Launches of the bucket kernels specialised on k.
template <bool FILL, int K>
int launch_hash_k(const HashParams &P, unsigned grid, int smem, int nt, cudaStream_t st) {
    if (nt == 512) {
        PROJ_CUDA_TRY(cudaFuncSetAttribute(hash_kernel<FILL, K, 512>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        hash_kernel<FILL, K, 512><<<grid, 512, smem, st>>>(P);
    } else {
        PROJ_CUDA_TRY(cudaFuncSetAttribute(hash_kernel<FILL, K, kThreads>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        hash_kernel<FILL, K, kThreads><<<grid, kThreads, smem, st>>>(P);
    }
    PROJ_LAUNCH_CHECK(FILL ? "hash_kernel<fill>" : "hash_kernel<count>");
    return PROJ_OK;
}

// nt: threads per CTA (1024, or 512 so that two or three units share an SM)
template <bool FILL>
int launch_hash(const HashParams &P, unsigned grid, int smem, cudaStream_t st, int nt = kThreads) {
    switch (P.k) {
        case 1: return launch_hash_k<FILL, 1>(P, grid, smem, nt, st);
        case 2: return launch_hash_k<FILL, 2>(P, grid, smem, nt, st);
        case 3: return launch_hash_k<FILL, 3>(P, grid, smem, nt, st);
        case 4: return launch_hash_k<FILL, 4>(P, grid, smem, nt, st);
        case 5: return launch_hash_k<FILL, 5>(P, grid, smem, nt, st);
        case 6: return launch_hash_k<FILL, 6>(P, grid, smem, nt, st);
        case 7: return launch_hash_k<FILL, 7>(P, grid, smem, nt, st);
        case 8: return launch_hash_k<FILL, 8>(P, grid, smem, nt, st);
        case 9: return launch_hash_k<FILL, 9>(P, grid, smem, nt, st);
        default: return launch_hash_k<FILL, 10>(P, grid, smem, nt, st);
    }
}

template <int K>
int launch_partition_k(const HashParams &P, dim3 grid, uint16_t *orel, uint16_t *olid,
                       int32_t *pstart, cudaStream_t st) {
    PROJ_CUDA_TRY(cudaFuncSetAttribute(part_sort_kernel<K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kSortSmem));
    {
        TraceSpan ts_("hash_partition", st);
        part_sort_kernel<K><<<grid, kSortThreads, kSortSmem, st>>>(P, orel, olid, pstart);
    }
    PROJ_LAUNCH_CHECK("part_sort_kernel");
    return PROJ_OK;
}

int launch_partition(const HashParams &P0, dim3 grid, uint16_t *orel, uint16_t *olid,
                     int32_t *pstart, int *info, cudaStream_t st) {
    HashParams P = P0;
    P.chunk_info = info;
    {
        TraceSpan ts_("hash_partition", st);
        chunk_info_kernel<<<(unsigned)((P.n_chunks + 127) / 128), 128, 0, st>>>(P, info);
    }
    PROJ_LAUNCH_CHECK("chunk_info_kernel");
    switch (P.k) {
        case 9: return launch_partition_k<9>(P, grid, orel, olid, pstart, st);
        case 10: return launch_partition_k<10>(P, grid, orel, olid, pstart, st);
        default: return launch_partition_k<0>(P, grid, orel, olid, pstart, st);
    }
}

// Capacity of each unit's enriched list: partitioned mode, the unit's l-mers
// over s; else a bound shared by all units.
__global__ void emit_cap_kernel(const int32_t *__restrict__ pstart, int n_chunks, int parts,
                                int64_t units, int s, int64_t uniform_cap,
                                int64_t *__restrict__ cap) {
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= units) return;
    if (!pstart) {
        cap[u] = uniform_cap;
        return;
    }
    const int64_t trial = u / parts;
    const int part = (int)(u % parts);
    const int32_t *ps = pstart + trial * n_chunks * (parts + 1);
    int64_t n = 0;
    for (int c = 0; c < n_chunks; ++c) n += ps[c * (parts + 1) + part + 1] - ps[c * (parts + 1) + part];
    cap[u] = n / s;
}

// Sizes of every enriched bucket from the counting pass's lists (no recount):
// unit u's entries go to cand_cnt[cand_base[u] ..] in key order.  A search that
// keeps only its largest buckets selects on these; the trials and keys of the
// kept ones come from the lists afterwards (kept_table_kernel).
__global__ void __launch_bounds__(256) hash_cnt_kernel(const HashParams P) {
    const int unit = blockIdx.x;
    const uint2 *src = P.emit + P.emit_off[unit];
    const int nb = P.part_nb[unit];
    const int64_t cb = P.cand_base[unit];
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (cb + i < P.cap_cand) P.cand_cnt[cb + i] = (int32_t)src[i].y;
}

// Trial and key of each kept candidate c = sel[i] (an index into the list of
// all enriched buckets): its unit is the last with cand_base <= c, its entry
// the (c - cand_base)-th of that unit's list.
__global__ void kept_table_kernel(const int64_t *__restrict__ cbase, int64_t n_units,
                                  const int64_t *__restrict__ emit_off, const uint2 *__restrict__ emit,
                                  int parts, int hb, int64_t trial_begin,
                                  const int64_t *__restrict__ sel, int64_t n,
                                  int32_t *__restrict__ cand_trial, uint32_t *__restrict__ cand_key) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t c = sel[i];
    int64_t lo = 0, hi = n_units - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (cbase[mid] <= c) lo = mid; else hi = mid - 1;
    }
    const uint2 e = emit[emit_off[lo] + (c - cbase[lo])];
    cand_trial[c] = (int32_t)(trial_begin + lo / parts);
    cand_key[c] = (uint32_t)(lo % parts) * (uint32_t)hb + e.x;
}

// Members of selected candidates (one CTA each), ascending: the l-mers of the
// candidate's trial whose projected key is the candidate's, compacted in
// l-mer order with ballot scans.  Partitioned mode scans the (trial, part)
// segment of the partition; otherwise every l-mer of the trial is rehashed.
__global__ void __launch_bounds__(kThreads) gather_sel_kernel(
    const HashParams P, const int64_t *__restrict__ sel, const int32_t *__restrict__ cand_trial,
    const uint32_t *__restrict__ cand_key, const int64_t *__restrict__ new_off,
    int32_t *__restrict__ out) {
    extern __shared__ __align__(16) uint8_t g_smem[];  // partitioned: the unit's chunk walk
    __shared__ int s_pos[16];
    __shared__ int s_round[kWarps + 1];
    __shared__ int2 s_warp[kWarps + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t ci = sel[blockIdx.x];
    const int trial_local = (int)(cand_trial[ci] - P.trial_begin);
    const uint32_t key = cand_key[ci];
    const uint32_t part = key / (uint32_t)P.hb, rel = key - part * (uint32_t)P.hb;
    const int64_t o0 = new_off[blockIdx.x], len = new_off[blockIdx.x + 1] - o0;
    int32_t *s_cb = reinterpret_cast<int32_t *>(g_smem);
    long long *s_pb = reinterpret_cast<long long *>(g_smem + (((P.n_chunks + 1) * 4 + 15) & ~15));
    int64_t n_iter;
    if (P.partitioned) {
        unit_walk_setup(P, trial_local, (int)part, s_cb, s_pb, s_warp);
        n_iter = s_cb[P.n_chunks];
        // Warp w takes the unit's entries [w W, w W + W) in rounds of 32, eight
        // rounds' loads in flight; an entry matches when its key is the
        // bucket's.  A first walk counts each warp's matches, a scan places the
        // warps, and a second walk writes the matches' l-mer ids in entry order
        // (the unit's entries are in l-mer order), ranked by ballots.
        const unsigned below = (1u << lane) - 1u;
        const int W = (int)(((n_iter + kWarps - 1) / kWarps + 31) & ~31);
        const int f0 = min((int)n_iter, warp * W), f1 = min((int)n_iter, f0 + W);
        auto walk = [&](bool write, int64_t at) {
            int cnt = 0, c = 0;
            for (int fb = f0; fb < f1; fb += 8 * 32) {
                uint32_t rv[8];
                int cc[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int f = fb + 32 * u + lane;
                    rv[u] = 0xFFFFFFFFu;
                    cc[u] = 0;
                    if (f < f1) {
                        while (s_cb[c + 1] <= f) ++c;
                        cc[u] = c;
                        rv[u] = P.prel[s_pb[c] + f];
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const bool e = rv[u] == rel;
                    const uint32_t bal = __ballot_sync(0xffffffffu, e);
                    if (write && e) {
                        const int f = fb + 32 * u + lane;
                        const int64_t q = at + cnt + __popc(bal & below);
                        if (q < len) out[o0 + q] = cc[u] * kSortChunk + (int)P.plid[s_pb[cc[u]] + f];
                    }
                    cnt += __popc(bal);
                }
            }
            return cnt;
        };
        const int found = walk(false, 0);
        if (lane == 0) s_round[warp] = found;
        __syncthreads();
        if (warp == 0) {
            const int v = lane < kWarps ? s_round[lane] : 0;
            int sc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, sc, o);
                if (lane >= o) sc += u;
            }
            if (lane < kWarps) s_round[lane] = sc - v;
        }
        __syncthreads();
        walk(true, s_round[warp]);
        return;
    } else {
        n_iter = P.x;
        trial_positions(P, trial_local, s_pos);
        __syncthreads();
    }
    int pos[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) pos[q] = q < P.k ? s_pos[q] : 0;
    int i = 0;
    int64_t running = 0;
    for (int64_t base = 0; base < n_iter; base += kThreads) {
        const int64_t it = base + tid;
        bool e = false;
        int gid = 0;
        if (it < n_iter) {
            gid = (int)it;
            while (__ldg(P.lmer_off + i + 1) <= gid) ++i;
            const int64_t b0 = (int64_t)__ldg(P.seq_off + i) + (gid - __ldg(P.lmer_off + i));
            e = lmer_key(window64(P.packed, P.nwords, b0), pos, P.k) == key;
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, e);
        if (lane == 0) s_round[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {
            const int v = lane < kWarps ? s_round[lane] : 0;
            int sc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, sc, o);
                if (lane >= o) sc += u;
            }
            if (lane < kWarps) s_round[lane] = sc - v;
            if (lane == kWarps - 1) s_round[kWarps] = sc;
        }
        __syncthreads();
        if (e) {
            const int64_t q = running + s_round[warp] + __popc(bal & ((1u << lane) - 1u));
            if (q < len) out[o0 + q] = gid;
        }
        running += s_round[kWarps];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Hash-tile autotuning: the bucket kernels run as 1024-thread CTAs or, when a
// unit's shared memory lets several share an SM, as 512-thread CTAs.  The first
// search of each shape class (k, counter layout, parts, ceil(log2) of l-mers and
// of units, sequences) times its counting pass both ways on its own data (the
// pass is idempotent) and keeps the faster for both passes (per process);
// PROJ_AUTOTUNE=0 keeps 1024 and PROJ_HASH_NT=512|1024 forces one.
// ---------------------------------------------------------------------------
std::mutex g_hash_tune_mu;
std::map<uint64_t, int> g_hash_tuned;

uint64_t hash_shape_key(const HashParams &P, int64_t n_units) {
    int xb = 0, ub = 0;
    while (((int64_t)1 << xb) < (int64_t)P.x) ++xb;
    while (((int64_t)1 << ub) < n_units) ++ub;
    return ((uint64_t)P.k << 56) | ((uint64_t)P.hist16 << 55) | ((uint64_t)P.parts << 48) |
           ((uint64_t)xb << 40) | ((uint64_t)ub << 32) | (uint64_t)std::min(P.t, 1 << 20);
}

// 0 = not decided (tune), else the CTA size to use
int hash_nt_choice(const HashParams &P, int64_t n_units, int fill_smem) {
    if (P.partitioned || fill_smem > 113 * 1024) return kThreads;  // one unit per SM anyway
    if (const char *f = getenv("PROJ_HASH_NT")) {
        const int v = atoi(f);
        if (v == 512 || v == 1024) return v;
    }
    const char *env = getenv("PROJ_AUTOTUNE");
    if (env && env[0] == '0') return kThreads;
    std::lock_guard<std::mutex> lk(g_hash_tune_mu);
    auto it = g_hash_tuned.find(hash_shape_key(P, n_units));
    return it == g_hash_tuned.end() ? 0 : it->second;
}

}  // namespace

int run_trial_hash(const uint32_t *packed, const Layout &L, int k, int s, uint64_t seed,
                   int64_t trial_begin, int64_t n_trials, const int32_t *positions_in,
                   const HashOut &out, cudaStream_t st) {
    PROJ_REQUIRE(k >= 1 && k <= 10 && k <= L.l, "need 1 <= k <= min(l, 10), got k=%d l=%d", k, L.l);
    PROJ_REQUIRE(s >= 1, "need s >= 1, got %d", s);
    PROJ_REQUIRE(n_trials >= 0 && n_trials <= (int64_t)1 << 24, "n_trials out of range");
    PROJ_REQUIRE(trial_begin >= 0, "trial_begin must be >= 0");
    PROJ_REQUIRE(out.totals != nullptr, "totals_dev must not be NULL");
    PROJ_REQUIRE(out.cap_cand >= 0 && out.cap_members >= 0, "capacities must be >= 0");
    PROJ_REQUIRE(out.cap_cand == 0 || (out.cand_trial && out.cand_key && out.cand_cnt),
                 "candidate buffers must not be NULL");
    PROJ_REQUIRE(out.cand_off != nullptr, "cand_off_dev must not be NULL");
    PROJ_REQUIRE(out.cap_members == 0 || out.members, "members_dev must not be NULL");

    HashParams P{};
    P.packed = packed;
    P.nwords = L.nwords;
    P.seq_off = L.seq_off_dev();
    P.lmer_off = L.lmer_off_dev();
    P.t = L.t; P.l = L.l; P.k = k; P.s = s; P.x = (int)L.x;
    P.seed = seed;
    P.trial_begin = trial_begin;
    const int64_t nbuck = (int64_t)1 << (2 * k);
    // u32 counters when they fit; else u16 pairs if no bucket can pass 65535
    if (nbuck * 4 <= kHistBytes) {
        P.hist16 = 0; P.hb = (int)nbuck; P.parts = 1;
    } else if (L.x <= 65535) {
        P.hist16 = 1; P.hb = (int)std::min<int64_t>(nbuck, kHistBytes / 2); P.parts = (int)(nbuck / P.hb);
    } else {
        P.hist16 = 0; P.hb = kHistBytes / 4; P.parts = (int)(nbuck / P.hb);
    }
    if (positions_in) {
        P.fixed_pos = 1;
        for (int q = 0; q < k; ++q) {
            PROJ_REQUIRE(positions_in[q] >= 0 && positions_in[q] < L.l &&
                             (q == 0 || positions_in[q] > positions_in[q - 1]),
                         "positions_in must be increasing and in [0, l)");
            P.pos_in[q] = positions_in[q];
        }
    }
    P.pos_out = out.positions;
    P.counts_out = out.counts;
    // stage the packed input when it fits next to the histogram (the
    // partitioned mode reads precomputed keys instead)
    const bool partitioned = P.parts > 1 && L.x > 65535;
    if (partitioned) {
        P.partitioned = 1;
        PROJ_REQUIRE(P.hb == (int)kPartKeys && !P.hist16, "partitioned mode expects u32 parts");
        P.count16 = 1;  // the counting pass in 64 KB (two units per SM)
        P.n_chunks = (int)((L.x + kSortChunk - 1) / kSortChunk);
        PROJ_REQUIRE(P.n_chunks <= kMaxSortChunks,
                     "%lld l-mers exceed the partitioned mode's %d chunks of %d",
                     (long long)L.x, kMaxSortChunks, kSortChunk);
    } else {
        HashParams Q = P;
        Q.stage_words = (int)L.nwords;
        if (smem_layout(Q, true).total <= kSmemLimit) P.stage_words = (int)L.nwords;
    }
    const SmemLayout S1 = smem_layout(P, false), S2 = smem_layout(P, true);
    PROJ_REQUIRE(S2.total <= kSmemLimit, "too many sequences for the shared-memory layout (t=%d)", L.t);

    const int64_t n_units = n_trials * P.parts;
    if (n_units == 0) {
        PROJ_CUDA_TRY(cudaMemsetAsync(out.totals, 0, 2 * sizeof(int64_t), st));
        PROJ_CUDA_TRY(cudaMemcpyAsync(out.cand_off, out.totals, sizeof(int64_t),
                                      cudaMemcpyDeviceToDevice, st));
        return PROJ_OK;
    }
    PROJ_REQUIRE(n_units < (int64_t)1 << 31, "too many (trial, part) units");
    const bool reuse = out.state && out.state->valid;
    // every trial's positions drawn once for all of this call's kernels (and the
    // filling call and member gather of the same search)
    DevBuf pos_own;  // freed (stream-ordered) after this call's launches
    if (!P.fixed_pos) {
        DevBuf &pos_buf = out.state ? out.state->pos_buf : pos_own;
        if (!reuse) {
            PROJ_TRY(pos_buf.alloc((size_t)n_trials * k, st));
            PROJ_TRY(launch_positions(seed, trial_begin, n_trials, L.l, k, pos_buf.as<uint8_t>(), st));
        }
        P.pos_tab = pos_buf.as<uint8_t>();
    }
    DevBuf meta_own, part_own;
    DevBuf &meta = out.state ? out.state->meta : meta_own;
    DevBuf &part_buf = out.state ? out.state->part_buf : part_own;
    if (!reuse) PROJ_TRY(meta.alloc((size_t)n_units * (4 + 4 + 8 + 8), st));
    P.part_nb = meta.as<int32_t>();
    P.part_nm = P.part_nb + n_units;
    int64_t *cbase = reinterpret_cast<int64_t *>(P.part_nm + n_units);
    int64_t *mbase = cbase + n_units;
    P.cand_base = cbase;
    P.mem_base = mbase;

    // large inputs over several key-range parts: group each trial's keys by
    // part first.  part_buf: [part starts (int32) | keys (u16) | chunk-local ids (u16)]
    if (partitioned) {
        PROJ_REQUIRE(P.parts <= kMaxParts, "too many key-range parts");
        const int64_t n_pst = n_trials * P.n_chunks * (P.parts + 1);
        const int64_t n_ent = n_trials * P.n_chunks * kSortChunk;
        if (!reuse)
            PROJ_TRY(part_buf.alloc((size_t)n_pst * 4 + 16 + (size_t)n_ent * 4 +
                                        (size_t)P.n_chunks * 32, st));
        int32_t *pst = part_buf.as<int32_t>();
        uint16_t *rel = reinterpret_cast<uint16_t *>(
            (reinterpret_cast<uintptr_t>(pst + n_pst) + 15) & ~(uintptr_t)15);
        P.pstart = pst;
        P.prel = rel;
        P.plid = rel + n_ent;
        if (!reuse) {
            const dim3 grid((unsigned)P.n_chunks, (unsigned)n_trials);
            int *info = reinterpret_cast<int *>(rel + 2 * n_ent);  // [n_chunks][8]
            PROJ_TRY(launch_partition(P, grid, rel, rel + n_ent, pst, info, st));
        }
    }
    // each unit's enriched (key, size) list kept by the counting pass (a search
    // that keeps only its largest buckets builds its table from them)
    HashState *hs = out.state;
    if (hs && out.want_emit && !reuse) {
        const int64_t cap_u = std::min<int64_t>(P.hb, L.x / s);
        const int64_t ub = partitioned ? n_trials * L.x / s + n_units : n_units * cap_u;
        PROJ_TRY(hs->emit_buf.alloc((size_t)(2 * n_units + 1) * 8 + (size_t)ub * 8, st));
        int64_t *eoff = hs->emit_buf.as<int64_t>();
        int64_t *ecap = eoff + n_units + 1;
        emit_cap_kernel<<<(unsigned)((n_units + 255) / 256), 256, 0, st>>>(
            partitioned ? P.pstart : nullptr, P.n_chunks, P.parts, n_units, s, cap_u, ecap);
        PROJ_LAUNCH_CHECK("emit_cap_kernel");
        scan_i64_kernel<<<1, 1024, 0, st>>>(ecap, n_units, eoff);
        PROJ_LAUNCH_CHECK("scan_i64_kernel");
        hs->emitted = true;
    }
    if (hs && hs->emitted) {
        P.emit_off = hs->emit_buf.as<int64_t>();
        P.emit = reinterpret_cast<uint2 *>(hs->emit_buf.as<int64_t>() + 2 * n_units + 1);
    }
    if (hs) {
        hs->parts = P.parts;
        if (!reuse) hs->nt = 0;  // set once the counting pass has chosen
        hs->hb = P.hb;
        hs->n_chunks = P.n_chunks;
        hs->partitioned = partitioned;
        hs->prel = P.prel;
        hs->plid = P.plid;
        hs->pstart = P.pstart;
        hs->pos_tab = P.pos_tab;
    }
    int nt = hs && reuse ? hs->nt : hash_nt_choice(P, n_units, S2.total);
    if (nt == 0 && !hs) nt = kThreads;  // plain calls do not synchronise to tune
    if (!reuse) {
        if (nt == 0) {
            // time the (idempotent) counting pass with both CTA sizes, keep the faster
            cudaEvent_t e[3];
            for (int q = 0; q < 3; ++q) PROJ_CUDA_TRY(cudaEventCreate(&e[q]));
            PROJ_CUDA_TRY(cudaEventRecord(e[0], st));
            {
                TraceSpan ts_("hash_count", st);
                PROJ_TRY(launch_hash<false>(P, (unsigned)n_units, S1.total, st, kThreads));
            }
            PROJ_CUDA_TRY(cudaEventRecord(e[1], st));
            PROJ_TRY(launch_hash<false>(P, (unsigned)n_units, S1.total, st, 512));
            PROJ_CUDA_TRY(cudaEventRecord(e[2], st));
            PROJ_CUDA_TRY(cudaEventSynchronize(e[2]));
            float t1024 = 0.f, t512 = 0.f;
            PROJ_CUDA_TRY(cudaEventElapsedTime(&t1024, e[0], e[1]));
            PROJ_CUDA_TRY(cudaEventElapsedTime(&t512, e[1], e[2]));
            for (int q = 0; q < 3; ++q) cudaEventDestroy(e[q]);
            nt = t512 < 0.97f * t1024 ? 512 : kThreads;
            std::lock_guard<std::mutex> lk(g_hash_tune_mu);
            g_hash_tuned[hash_shape_key(P, n_units)] = nt;
        } else {
            // a partitioned counting pass runs two 512-thread units per SM
            // (measured: 1024 threads, one unit per SM, 24% slower; 256 threads 6%)
            int cnt_nt = nt;
            if (P.count16) {
                cnt_nt = 512;
                if (const char *f = getenv("PROJ_HASH_NT"))
                    if (atoi(f) == 1024) cnt_nt = 1024;
            }
            TraceSpan ts_("hash_count", st);
            PROJ_TRY(launch_hash<false>(P, (unsigned)n_units, S1.total, st, cnt_nt));
        }
        {
            TraceSpan ts_("hash_scan", st);
            hash_scan_kernel<<<1, 1024, 0, st>>>(P.part_nb, P.part_nm, (int)n_units, cbase, mbase,
                                                 out.totals, out.cap_cand, out.cand_off);
        }
        PROJ_LAUNCH_CHECK("hash_scan_kernel");
    } else {
        // the counting call wrote the totals; only the end of the offsets is new
        cand_end_kernel<<<1, 1, 0, st>>>(out.totals, out.cap_cand, out.cand_off);
        PROJ_LAUNCH_CHECK("cand_end_kernel");
    }
    if (hs) hs->nt = nt;  // the filling call of this search uses the same CTA size
    if (out.count_only) {
        if (out.state) out.state->valid = true;
        return PROJ_OK;
    }
    P.cap_cand = out.cap_cand;
    P.cand_trial = out.cand_trial;
    P.cand_key = out.cand_key;
    P.cand_cnt = out.cand_cnt;
    P.cand_off = out.cand_off;
    if (out.table_only) {
        PROJ_REQUIRE(reuse && hs && hs->emitted, "a table-only fill needs the counting call's lists");
        {
            TraceSpan ts_("hash_table", st);
            hash_cnt_kernel<<<(unsigned)n_units, 256, 0, st>>>(P);
        }
        PROJ_LAUNCH_CHECK("hash_cnt_kernel");
        hs->n_units = n_units;
        hs->trial_begin = trial_begin;
        hs->cand_base = cbase;
        return PROJ_OK;
    }
    P.emit = nullptr;

    DevBuf scratch;
    if (out.cap_members > 0) PROJ_TRY(scratch.alloc((size_t)out.cap_members * 8, st));
    P.cap_cand = out.cap_cand;
    P.cap_members = out.cap_members;
    P.cand_trial = out.cand_trial;
    P.cand_key = out.cand_key;
    P.cand_cnt = out.cand_cnt;
    P.cand_off = out.cand_off;
    P.members = out.members;
    P.scratch_key = scratch.as<uint32_t>();
    P.scratch_gid = reinterpret_cast<int32_t *>(P.scratch_key + out.cap_members);
    P.counts_out = nullptr;
    P.pos_out = nullptr;
    {
        TraceSpan ts_("hash_fill", st);
        PROJ_TRY(launch_hash<true>(P, (unsigned)n_units, S2.total, st, nt));
    }
    return PROJ_OK;
}

int run_kept_table(const HashState &hs, const int64_t *sel, int64_t n, int32_t *cand_trial,
                   uint32_t *cand_key, cudaStream_t st) {
    PROJ_REQUIRE(hs.valid && hs.emitted && hs.cand_base, "the kept table needs the counting call's lists");
    if (n == 0) return PROJ_OK;
    const int64_t *eoff = hs.emit_buf.as<int64_t>();
    const uint2 *emit = reinterpret_cast<const uint2 *>(eoff + 2 * hs.n_units + 1);
    {
        TraceSpan ts_("hash_table", st);
        kept_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            hs.cand_base, hs.n_units, eoff, emit, hs.parts, hs.hb, hs.trial_begin, sel, n, cand_trial,
            cand_key);
    }
    PROJ_LAUNCH_CHECK("kept_table_kernel");
    return PROJ_OK;
}

int run_gather_members(const uint32_t *packed, const Layout &L, const HashState &hs, int k,
                       uint64_t seed, const int64_t *sel, int64_t n, const int32_t *cand_trial,
                       const uint32_t *cand_key, const int64_t *new_off, int32_t *new_members,
                       cudaStream_t st) {
    PROJ_REQUIRE(hs.valid && hs.hb > 0, "the member gather needs the counting call's state");
    if (n == 0) return PROJ_OK;
    HashParams P{};
    P.packed = packed;
    P.nwords = L.nwords;
    P.seq_off = L.seq_off_dev();
    P.lmer_off = L.lmer_off_dev();
    P.t = L.t; P.l = L.l; P.k = k; P.x = (int)L.x;
    P.seed = seed;
    P.trial_begin = 0;
    P.parts = hs.parts;
    P.hb = hs.hb;
    P.n_chunks = hs.n_chunks;
    P.pos_tab = hs.pos_tab;
    int smem = 0;
    if (hs.partitioned) {
        P.partitioned = 1;
        P.prel = hs.prel;
        P.plid = hs.plid;
        P.pstart = hs.pstart;
        smem = (((P.n_chunks + 1) * 4 + 15) & ~15) + P.n_chunks * 8;
    }
    PROJ_CUDA_TRY(cudaFuncSetAttribute(gather_sel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       std::max(smem, 1)));
    {
        TraceSpan ts_("hash_gather", st);
        gather_sel_kernel<<<(unsigned)n, kThreads, smem, st>>>(P, sel, cand_trial, cand_key, new_off,
                                                              new_members);
    }
    PROJ_LAUNCH_CHECK("gather_sel_kernel");
    return PROJ_OK;
}

namespace {

// per-instance candidate and member offsets: the scanned bases at each
// instance's first unit, and the totals at the end
__global__ void batch_begins_kernel(const int64_t *__restrict__ cbase,
                                    const int64_t *__restrict__ mbase,
                                    const int64_t *__restrict__ unit_begin, int n_inst,
                                    const int64_t *__restrict__ totals, int64_t *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_inst) {
        out[2 * i] = cbase[unit_begin[i]];
        out[2 * i + 1] = mbase[unit_begin[i]];
    } else if (i == n_inst) {
        out[2 * i] = totals[0];
        out[2 * i + 1] = totals[1];
    }
}

}  // namespace

int run_hash_batch(const std::vector<HashInstSpec> &spec, HashBatchOut &out, cudaStream_t st) {
    const int n = (int)spec.size();
    PROJ_REQUIRE(n >= 1, "empty batch");
    std::vector<HashParams> hp(n);
    std::vector<int64_t> unit_begin(n + 1, 0);
    int dyn1 = 0, dyn2 = 0;
    for (int i = 0; i < n; ++i) {
        const HashInstSpec &q = spec[i];
        PROJ_REQUIRE(q.k >= 1 && q.k <= 10 && q.k <= q.l, "instance %d: need 1 <= k <= min(l, 10)", i);
        PROJ_REQUIRE(q.s >= 1 && q.m >= 1, "instance %d: need s >= 1 and m >= 1", i);
        HashParams &P = hp[i];
        P = HashParams{};
        P.packed = q.packed;
        P.nwords = q.nwords;
        P.seq_off = q.seq_off_rel;
        P.lmer_off = q.lmer_off;
        P.t = q.t; P.l = q.l; P.k = q.k; P.s = q.s; P.x = q.x;
        P.seed = q.seed;
        P.trial_begin = 0;
        const int64_t nbuck = (int64_t)1 << (2 * q.k);
        if (nbuck * 4 <= kHistBytes) {
            P.hist16 = 0; P.hb = (int)nbuck; P.parts = 1;
        } else if (q.x <= 65535) {
            P.hist16 = 1; P.hb = (int)std::min<int64_t>(nbuck, kHistBytes / 2); P.parts = (int)(nbuck / P.hb);
        } else {
            P.hist16 = 0; P.hb = kHistBytes / 4; P.parts = (int)(nbuck / P.hb);
        }
        HashParams Q = P;
        Q.stage_words = (int)q.nwords;
        if (smem_layout(Q, true).total <= kSmemLimit) P.stage_words = (int)q.nwords;
        PROJ_REQUIRE(smem_layout(P, true).total <= kSmemLimit, "instance %d: too many sequences", i);
        dyn1 = std::max(dyn1, smem_layout(P, false).total);
        dyn2 = std::max(dyn2, smem_layout(P, true).total);
        unit_begin[i + 1] = unit_begin[i] + (int64_t)q.m * P.parts;
    }
    const int64_t U = unit_begin[n];
    PROJ_REQUIRE(U < ((int64_t)1 << 31), "too many (trial, part) units in the batch");

    DevBuf meta, ub, hpb, begins;
    PROJ_TRY(meta.alloc((size_t)U * (4 + 4 + 8 + 8), st));
    PROJ_TRY(ub.alloc((size_t)(n + 1) * sizeof(int64_t), st));
    PROJ_TRY(hpb.alloc((size_t)n * sizeof(HashParams), st));
    PROJ_TRY(begins.alloc((size_t)(n + 1) * 2 * sizeof(int64_t), st));
    int32_t *part_nb = meta.as<int32_t>();
    int32_t *part_nm = part_nb + U;
    int64_t *cbase = reinterpret_cast<int64_t *>(part_nm + U);
    int64_t *mbase = cbase + U;
    for (int i = 0; i < n; ++i) {
        HashParams &P = hp[i];
        P.part_nb = part_nb + unit_begin[i];
        P.part_nm = part_nm + unit_begin[i];
        P.cand_base = cbase + unit_begin[i];
        P.mem_base = mbase + unit_begin[i];
    }
    PROJ_CUDA_TRY(cudaMemcpyAsync(ub.as<int64_t>(), unit_begin.data(), (n + 1) * sizeof(int64_t),
                                  cudaMemcpyHostToDevice, st));
    PROJ_CUDA_TRY(cudaMemcpyAsync(hpb.as<HashParams>(), hp.data(), n * sizeof(HashParams),
                                  cudaMemcpyHostToDevice, st));
    PROJ_CUDA_TRY(cudaFuncSetAttribute(hash_batch_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
    PROJ_CUDA_TRY(cudaFuncSetAttribute(hash_batch_kernel<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
    {
        TraceSpan ts_("hash_count", st);
        hash_batch_kernel<false><<<(unsigned)U, kThreads, dyn1, st>>>(hpb.as<HashParams>(),
                                                                     ub.as<int64_t>(), n);
    }
    PROJ_LAUNCH_CHECK("hash_batch_kernel<count>");
    DevBuf tot;
    PROJ_TRY(tot.alloc(3 * sizeof(int64_t), st));
    int64_t *totals = tot.as<int64_t>();
    int64_t *off0 = totals + 2;  // sentinel slot (capacity 0 here)
    {
        TraceSpan ts_("hash_scan", st);
        hash_scan_kernel<<<1, 1024, 0, st>>>(part_nb, part_nm, (int)U, cbase, mbase, totals, 0, off0);
    }
    PROJ_LAUNCH_CHECK("hash_scan_kernel");
    batch_begins_kernel<<<(n + 1 + 255) / 256, 256, 0, st>>>(cbase, mbase, ub.as<int64_t>(), n,
                                                              totals, begins.as<int64_t>());
    PROJ_LAUNCH_CHECK("batch_begins_kernel");
    std::vector<int64_t> bh(2 * (n + 1));
    PROJ_CUDA_TRY(cudaMemcpyAsync(bh.data(), begins.as<int64_t>(), bh.size() * sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, st));
    PROJ_CUDA_TRY(cudaStreamSynchronize(st));
    out.C = bh[2 * n];
    out.M = bh[2 * n + 1];
    out.cand_begin.resize(n);
    out.n_cand.resize(n);
    out.mem_begin.resize(n);
    out.n_mem.resize(n);
    for (int i = 0; i < n; ++i) {
        out.cand_begin[i] = bh[2 * i];
        out.mem_begin[i] = bh[2 * i + 1];
        out.n_cand[i] = bh[2 * (i + 1)] - bh[2 * i];
        out.n_mem[i] = bh[2 * (i + 1) + 1] - bh[2 * i + 1];
    }
    const int64_t C = out.C, M = out.M;
    PROJ_TRY(out.cand.alloc((size_t)(C + 1) * 8 + (size_t)C * 12 + (size_t)M * 4 + 64, st));
    PROJ_CUDA_TRY(cudaMemcpyAsync(out.cand_off() + C, totals + 1, sizeof(int64_t),
                                  cudaMemcpyDeviceToDevice, st));
    DevBuf scratch;
    if (M > 0) PROJ_TRY(scratch.alloc((size_t)M * 8, st));
    for (int i = 0; i < n; ++i) {
        HashParams &P = hp[i];
        P.cap_cand = C;
        P.cap_members = M;
        P.cand_trial = out.cand_trial();
        P.cand_key = out.cand_key();
        P.cand_cnt = out.cand_cnt();
        P.cand_off = out.cand_off();
        P.members = out.members();
        P.scratch_key = scratch.as<uint32_t>();
        P.scratch_gid = reinterpret_cast<int32_t *>(P.scratch_key + M);
    }
    PROJ_CUDA_TRY(cudaMemcpyAsync(hpb.as<HashParams>(), hp.data(), n * sizeof(HashParams),
                                  cudaMemcpyHostToDevice, st));
    {
        TraceSpan ts_("hash_fill", st);
        hash_batch_kernel<true><<<(unsigned)U, kThreads, dyn2, st>>>(hpb.as<HashParams>(),
                                                                    ub.as<int64_t>(), n);
    }
    PROJ_LAUNCH_CHECK("hash_batch_kernel<fill>");
    return PROJ_OK;
}

}  // namespace proj

// ---------------------------------------------------------------------------
// trial_hash_noalloc: trial_hash without any device allocation.
//
// Some callers cannot call cudaMalloc: services that hand all device memory to
// their own pool allocator at start-up and forbid further allocations, and
// latency-critical callers that must not pay for an allocation (cudaMalloc may
// synchronise the whole device).  For them this entry point runs the same two
// bucket-kernel passes as trial_hash, but keeps its scratch (sequence and
// l-mer offsets, per-(trial, part) counts and output offsets, and the ordered
// list of enriched l-mers) in a fixed array that lives in the library's device
// image.  Every GPU that loads the library holds that array until the process
// exits.
// ---------------------------------------------------------------------------

static __device__ __align__(256) unsigned char g_noalloc_scratch[PROJ_NOALLOC_SCRATCH_BYTES];

namespace proj {
namespace {

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64];  // device address of g_noalloc_scratch per device ordinal

// Looks up (once per device, with that device current) the device address of
// the scratch array.  In host code the array's name is only a host-side
// stand-in, so kernels must receive this address instead.  The cached address
// assumes the device's primary context lives as long as the process: after a
// cudaDeviceReset the module is loaded again and the cache would be stale.
int noalloc_scratch(void **out) {
    int dev = 0;
    PROJ_CUDA_TRY(cudaGetDevice(&dev));
    PROJ_REQUIRE(dev >= 0 && dev < 64, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        PROJ_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return PROJ_OK;
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

// The sequence and l-mer offsets travel to the scratch array inside kernel
// parameters (copied by value at launch), not by a copy from host memory, so
// nothing on the device refers to the caller's or this call's host buffers.
constexpr int kOffChunk = 992;  // int32 values per launch (parameters stay under 4 KB)
struct OffChunk {
    int32_t *dst;
    int n;
    int32_t v[kOffChunk];
};

__global__ void noalloc_offsets_kernel(const OffChunk c) {
    for (int i = threadIdx.x; i < c.n; i += blockDim.x) c.dst[i] = c.v[i];
}

}  // namespace
}  // namespace proj

using namespace proj;

extern "C" int trial_hash_noalloc(const uint32_t *packed_dev, const int64_t *seq_off, int t, int l,
                                  int k, int s, uint64_t seed, int64_t trial_begin,
                                  int64_t n_trials, const int32_t *positions_in,
                                  uint8_t *positions_out_dev, uint32_t *counts_out_dev,
                                  int64_t cap_cand, int64_t cap_members, int32_t *cand_trial_dev,
                                  uint32_t *cand_key_dev, int32_t *cand_cnt_dev,
                                  int64_t *cand_off_dev, int32_t *members_dev,
                                  int64_t *totals_dev, void *stream) {
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    PROJ_REQUIRE(packed_dev != nullptr && seq_off != nullptr, "NULL input");
    PROJ_REQUIRE(t >= 1 && l >= 1 && l <= 32, "need t >= 1 and 1 <= l <= 32");
    PROJ_REQUIRE(k >= 1 && k <= 10 && k <= l, "need 1 <= k <= min(l, 10), got k=%d l=%d", k, l);
    PROJ_REQUIRE(s >= 1, "need s >= 1, got %d", s);
    PROJ_REQUIRE(n_trials >= 0 && n_trials <= (int64_t)1 << 24 && trial_begin >= 0,
                 "trial range out of range");
    PROJ_REQUIRE(totals_dev && cand_off_dev, "totals_dev and cand_off_dev must not be NULL");
    PROJ_REQUIRE(cap_cand >= 0 && cap_members >= 0, "capacities must be >= 0");
    PROJ_REQUIRE(cap_cand == 0 || (cand_trial_dev && cand_key_dev && cand_cnt_dev),
                 "candidate buffers must not be NULL");
    PROJ_REQUIRE(cap_members == 0 || members_dev, "members_dev must not be NULL");
    PROJ_REQUIRE(seq_off[0] == 0, "seq_off[0] must be 0");

    // host-side offsets (no device allocation)
    std::vector<int32_t> off(2 * (size_t)(t + 1));
    int64_t x = 0;
    for (int i = 0; i < t; ++i) {
        const int64_t n = seq_off[i + 1] - seq_off[i];
        PROJ_REQUIRE(n >= l, "sequence %d has length %lld < l = %d", i, (long long)n, l);
        PROJ_REQUIRE(seq_off[i + 1] < ((int64_t)1 << 31), "input longer than 2^31 - 1 bases");
        off[i + 1] = (int32_t)seq_off[i + 1];
        x += n - l + 1;
        off[t + 1 + i + 1] = (int32_t)x;
    }
    off[0] = 0;
    off[t + 1] = 0;

    HashParams P{};
    P.packed = packed_dev;
    P.nwords = (seq_off[t] + 15) / 16;
    P.t = t; P.l = l; P.k = k; P.s = s; P.x = (int)x;
    P.seed = seed;
    P.trial_begin = trial_begin;
    const int64_t nbuck = (int64_t)1 << (2 * k);
    if (nbuck * 4 <= kHistBytes) {
        P.hist16 = 0; P.hb = (int)nbuck; P.parts = 1;
    } else if (x <= 65535) {
        P.hist16 = 1; P.hb = (int)std::min<int64_t>(nbuck, kHistBytes / 2); P.parts = (int)(nbuck / P.hb);
    } else {
        P.hist16 = 0; P.hb = kHistBytes / 4; P.parts = (int)(nbuck / P.hb);
    }
    if (positions_in) {
        P.fixed_pos = 1;
        for (int q = 0; q < k; ++q) {
            PROJ_REQUIRE(positions_in[q] >= 0 && positions_in[q] < l &&
                             (q == 0 || positions_in[q] > positions_in[q - 1]),
                         "positions_in must be increasing and in [0, l)");
            P.pos_in[q] = positions_in[q];
        }
    }
    P.pos_out = positions_out_dev;
    P.counts_out = counts_out_dev;
    {
        HashParams Q = P;
        Q.stage_words = (int)P.nwords;
        if (smem_layout(Q, true).total <= kSmemLimit) P.stage_words = (int)P.nwords;
    }
    const SmemLayout S1 = smem_layout(P, false), S2 = smem_layout(P, true);
    PROJ_REQUIRE(S2.total <= kSmemLimit, "too many sequences for the shared-memory layout (t=%d)", t);
    const int64_t n_units = n_trials * P.parts;

    // carve the fixed scratch array
    const size_t b_off = align256(off.size() * sizeof(int32_t));
    const size_t b_cnt = align256((size_t)n_units * 2 * sizeof(int32_t));
    const size_t b_base = align256((size_t)n_units * 2 * sizeof(int64_t));
    const size_t b_list = align256((size_t)cap_members * (sizeof(uint32_t) + sizeof(int32_t)));
    const size_t need = b_off + b_cnt + b_base + b_list;
    if (need > (size_t)PROJ_NOALLOC_SCRATCH_BYTES) {
        set_error("trial_hash_noalloc needs %zu bytes of scratch for t=%d, %lld trials x %d parts "
                  "and cap_members=%lld, above its fixed %u bytes; use fewer trials per call, a "
                  "smaller cap_members, or trial_hash",
                  need, t, (long long)n_trials, P.parts, (long long)cap_members,
                  (unsigned)PROJ_NOALLOC_SCRATCH_BYTES);
        return PROJ_ECAPACITY;
    }
    void *scr = nullptr;
    PROJ_TRY(noalloc_scratch(&scr));
    unsigned char *base = (unsigned char *)scr;
    int32_t *d_off = (int32_t *)base;
    P.seq_off = d_off;
    P.lmer_off = d_off + (t + 1);
    P.part_nb = (int32_t *)(base + b_off);
    P.part_nm = P.part_nb + n_units;
    int64_t *cbase = (int64_t *)(base + b_off + b_cnt);
    int64_t *mbase = cbase + n_units;
    P.cand_base = cbase;
    P.mem_base = mbase;
    P.scratch_key = (uint32_t *)(base + b_off + b_cnt + b_base);
    P.scratch_gid = (int32_t *)(P.scratch_key + cap_members);
    // every scratch word is written before it is read (offsets here, counts by
    // pass 1, bases by the scan, the list by pass 2), so nothing is cleared
    for (size_t b = 0; b < off.size(); b += kOffChunk) {
        OffChunk c;
        c.dst = d_off + b;
        c.n = (int)std::min<size_t>(kOffChunk, off.size() - b);
        std::copy(off.begin() + b, off.begin() + b + c.n, c.v);
        noalloc_offsets_kernel<<<1, 256, 0, st>>>(c);
        PROJ_LAUNCH_CHECK("noalloc_offsets_kernel");
    }

    if (n_units == 0) {
        PROJ_CUDA_TRY(cudaMemsetAsync(totals_dev, 0, 2 * sizeof(int64_t), st));
        PROJ_CUDA_TRY(cudaMemsetAsync(cand_off_dev, 0, sizeof(int64_t), st));
        return PROJ_OK;
    }
    {
        TraceSpan ts_("hash_count", st);
        PROJ_TRY(launch_hash<false>(P, (unsigned)n_units, S1.total, st));
    }
    {
        TraceSpan ts_("hash_scan", st);
        hash_scan_kernel<<<1, 1024, 0, st>>>(P.part_nb, P.part_nm, (int)n_units, cbase, mbase,
                                             totals_dev, cap_cand, cand_off_dev);
    }
    PROJ_LAUNCH_CHECK("hash_scan_kernel");
    P.cap_cand = cap_cand;
    P.cap_members = cap_members;
    P.cand_trial = cand_trial_dev;
    P.cand_key = cand_key_dev;
    P.cand_cnt = cand_cnt_dev;
    P.cand_off = cand_off_dev;
    P.members = members_dev;
    P.counts_out = nullptr;
    P.pos_out = nullptr;
    {
        TraceSpan ts_("hash_fill", st);
        PROJ_TRY(launch_hash<true>(P, (unsigned)n_units, S2.total, st));
    }
    return PROJ_OK;
}

// ---------------------------------------------------------------------------
// projection_hist_peak: the shared-memory histogram rate the bucket kernels
// are measured against.  Every CTA (1024 threads, one per SM) counts
// register-generated pseudo-random keys into a shared-memory histogram laid
// out as the bucket kernels lay out the 4^k buckets of one CTA (u32 counters
// when 4^k of them fit in 128 KB, else u16 pairs over 65,536 buckets).
// ---------------------------------------------------------------------------
namespace proj {
namespace {

__global__ void __launch_bounds__(kThreads, 1) hist_peak_kernel(uint32_t mask, int hist16, int iters,
                                                                 uint32_t *sink) {
    extern __shared__ uint32_t h[];
    const int words = hist16 ? (int)((mask + 1) / 2) : (int)(mask + 1);
    for (int w = threadIdx.x; w < words; w += kThreads) h[w] = 0u;
    __syncthreads();
    uint32_t x = 0x9E3779B9u * (blockIdx.x * kThreads + threadIdx.x + 1);
    for (int i = 0; i < iters; ++i) {
        x ^= x << 13;  // xorshift32 (Marsaglia 2003)
        x ^= x >> 17;
        x ^= x << 5;
        const uint32_t key = x & mask;
        if (hist16) atomicAdd(&h[key >> 1], 1u << (16 * (key & 1u)));
        else atomicAdd(&h[key], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) sink[blockIdx.x] = h[x & (uint32_t)(words - 1)];  // keep the work
}

}  // namespace
}  // namespace proj

extern "C" int projection_hist_peak(int k, double *updates_per_s, void *stream) {
    using namespace proj;
    clear_error();
    PROJ_REQUIRE(updates_per_s != nullptr, "updates_per_s must not be NULL");
    PROJ_REQUIRE(k >= 1 && k <= 10, "need 1 <= k <= 10");
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t nbuck = 1ull << (2 * k);
    const int hist16 = nbuck * 4 > (uint64_t)kHistBytes;
    const uint32_t mask = (uint32_t)(hist16 ? std::min<uint64_t>(nbuck, 65536) : nbuck) - 1u;
    const size_t smem = hist16 ? (size_t)(mask + 1) * 2 : (size_t)(mask + 1) * 4;
    const int grid = sm_count();
    const int iters = 16384;
    DevBuf sink;
    PROJ_TRY(sink.alloc((size_t)grid * 4, st));
    PROJ_CUDA_TRY(cudaFuncSetAttribute(hist_peak_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    cudaEvent_t e0, e1;
    PROJ_CUDA_TRY(cudaEventCreate(&e0));
    PROJ_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {  // first launch warms up; keep the fastest
        PROJ_CUDA_TRY(cudaEventRecord(e0, st));
        hist_peak_kernel<<<grid, kThreads, smem, st>>>(mask, hist16, iters, sink.as<uint32_t>());
        PROJ_CUDA_TRY(cudaEventRecord(e1, st));
        PROJ_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        PROJ_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    PROJ_LAUNCH_CHECK("hist_peak_kernel");
    *updates_per_s = (double)grid * kThreads * iters / (best * 1e-3);
    return PROJ_OK;
}
