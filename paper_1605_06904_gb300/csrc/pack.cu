// Step a1 (linear 2-bit input, Section 6), the background frequencies of the
// motif model's column 0 (Section 5.1), and the per-trial projection positions
// of Algorithm 2 step 2a.
#include <algorithm>

#include "common.cuh"

namespace proj {
namespace {

// One thread per output word: 16 ASCII bases -> 16 two-bit codes A0 C1 T2 G3.
// HBM-bound (1 byte read + 0.25 byte written per base).
__global__ void pack_kernel(const uint8_t *__restrict__ ascii, int64_t total,
                            uint32_t *__restrict__ packed,
                            unsigned long long *__restrict__ bad) {
    const int64_t nw = (total + 15) >> 4;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b0 = w << 4;
        const int nb = (int)(total - b0 < 16 ? total - b0 : 16);
        uint8_t ch[16];
        if (nb == 16 && ((reinterpret_cast<uintptr_t>(ascii + b0) & 15u) == 0)) {
            const uint4 v = *reinterpret_cast<const uint4 *>(ascii + b0);
            memcpy(ch, &v, 16);
        } else {
            for (int q = 0; q < 16; ++q) ch[q] = q < nb ? ascii[b0 + q] : (uint8_t)'A';
        }
        uint32_t word = 0u;
        int first_bad = -1;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const uint8_t u = ch[q] & 0xDFu;  // upper case
            uint32_t c;
            if (u == 'A') c = 0u;
            else if (u == 'C') c = 1u;
            else if (u == 'T') c = 2u;
            else if (u == 'G') c = 3u;
            else { c = 0u; if (first_bad < 0 && q < nb) first_bad = q; }
            if (q < nb) word |= c << (2 * q);
        }
        packed[w] = word;
        if (first_bad >= 0) atomicMin(bad, (unsigned long long)(b0 + first_bad));
    }
}

// Block-wide sums of three per-thread counts (warp shuffles, then warp order);
// the result is valid in thread 0.  blockDim.x is a multiple of 32.
__device__ __forceinline__ void block_sum3(unsigned long long &a, unsigned long long &b,
                                           unsigned long long &c) {
    __shared__ unsigned long long part[32][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) { part[warp][0] = a; part[warp][1] = b; part[warp][2] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = b = c = 0ull;
        for (int w = 0; w < nw; ++w) { a += part[w][0]; b += part[w][1]; c += part[w][2]; }
    }
}

// Base counts by popcount over packed words (single CTA; the input is a few
// MB at most for the workloads in scope).
__global__ void background_kernel(const uint32_t *__restrict__ packed, int64_t total,
                                  double *__restrict__ bg) {
    unsigned long long c1 = 0, c2 = 0, c3 = 0;  // C, T, G (A = rest)
    const int64_t nw = (total + 15) >> 4;
    for (int64_t w = threadIdx.x; w < nw; w += blockDim.x) {
        uint32_t v = packed[w];
        const int nb = (int)(total - (w << 4) < 16 ? total - (w << 4) : 16);
        const uint32_t valid = nb == 16 ? 0x55555555u : ((1u << (2 * nb)) - 1u) & 0x55555555u;
        const uint32_t lo = v & valid, hi = (v >> 1) & valid;
        c1 += __popc(lo & ~hi);
        c2 += __popc(hi & ~lo);
        c3 += __popc(lo & hi);
    }
    block_sum3(c1, c2, c3);
    if (threadIdx.x == 0) {
        unsigned long long c[4];
        c[1] = c1; c[2] = c2; c[3] = c3;
        c[0] = (unsigned long long)total - c[1] - c[2] - c[3];
        unsigned long long tot = 0;
        for (int a = 0; a < 4; ++a) { if (c[a] == 0) c[a] = 1; tot += c[a]; }
        for (int a = 0; a < 4; ++a) bg[a] = (double)c[a] / (double)tot;
    }
}

// Background of each instance of a batch: base counts over its base range
// [base_range[2i], base_range[2i+1]) of the packed input (one CTA each).
__global__ void background_batch_kernel(const uint32_t *__restrict__ packed,
                                        const int64_t *__restrict__ base_range,
                                        double *__restrict__ bg) {
    const int64_t b0 = base_range[2 * blockIdx.x], b1 = base_range[2 * blockIdx.x + 1];
    unsigned long long c1 = 0, c2 = 0, c3 = 0;
    for (int64_t w = (b0 >> 4) + threadIdx.x; w <= ((b1 - 1) >> 4); w += blockDim.x) {
        const int64_t lo = w << 4;
        const int first = (int)(b0 > lo ? b0 - lo : 0);            // first valid base in the word
        const int last = (int)(b1 - lo < 16 ? b1 - lo : 16);         // one past the last
        uint32_t valid = 0u;
        for (int q = first; q < last; ++q) valid |= 1u << (2 * q);
        const uint32_t v = packed[w];
        const uint32_t lo2 = v & valid, hi2 = (v >> 1) & valid;
        c1 += __popc(lo2 & ~hi2);
        c2 += __popc(hi2 & ~lo2);
        c3 += __popc(lo2 & hi2);
    }
    block_sum3(c1, c2, c3);
    if (threadIdx.x == 0) {
        unsigned long long c[4];
        c[1] = c1; c[2] = c2; c[3] = c3;
        c[0] = (unsigned long long)(b1 - b0) - c[1] - c[2] - c[3];
        unsigned long long tot = 0;
        for (int a = 0; a < 4; ++a) { if (c[a] == 0) c[a] = 1; tot += c[a]; }
        for (int a = 0; a < 4; ++a) bg[4 * blockIdx.x + a] = (double)c[a] / (double)tot;
    }
}

__global__ void positions_kernel(uint64_t seed, int64_t trial_begin, int64_t n_trials, int l,
                                 int k, uint8_t *__restrict__ pos) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_trials) return;
    int p[32];
    draw_positions(seed, (uint64_t)(trial_begin + i), l, k, p);
    for (int q = 0; q < k; ++q) pos[i * k + q] = (uint8_t)p[q];
}

}  // namespace

int launch_pack(const uint8_t *ascii, int64_t total, uint32_t *packed, int64_t *bad,
                cudaStream_t st) {
    PROJ_CUDA_TRY(cudaMemsetAsync(bad, 0xFF, sizeof(int64_t), st));
    if (total == 0) return PROJ_OK;
    const int64_t nw = (total + 15) >> 4;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((nw + threads - 1) / threads, (int64_t)sm_count() * 8);
    {
        TraceSpan ts_("pack", st);
        pack_kernel<<<(unsigned)blocks, threads, 0, st>>>(
            ascii, total, packed, reinterpret_cast<unsigned long long *>(bad));
    }
    PROJ_LAUNCH_CHECK("pack_kernel");
    return PROJ_OK;
}

int launch_background(const uint32_t *packed, int64_t total, double *bg, cudaStream_t st) {
    {
        TraceSpan ts_("background", st);
        background_kernel<<<1, 1024, 0, st>>>(packed, total, bg);
    }
    PROJ_LAUNCH_CHECK("background_kernel");
    return PROJ_OK;
}

int launch_background_batch(const uint32_t *packed, const int64_t *base_range, int n_inst,
                            double *bg, cudaStream_t st) {
    {
        TraceSpan ts_("background", st);
        background_batch_kernel<<<n_inst, 256, 0, st>>>(packed, base_range, bg);
    }
    PROJ_LAUNCH_CHECK("background_batch_kernel");
    return PROJ_OK;
}

int launch_positions(uint64_t seed, int64_t trial_begin, int64_t n_trials, int l, int k,
                     uint8_t *pos, cudaStream_t st) {
    if (n_trials <= 0) return PROJ_OK;
    const int threads = 128;
    {
        TraceSpan ts_("positions", st);
        positions_kernel<<<(unsigned)((n_trials + threads - 1) / threads), threads, 0, st>>>(
            seed, trial_begin, n_trials, l, k, pos);
    }
    PROJ_LAUNCH_CHECK("positions_kernel");
    return PROJ_OK;
}

}  // namespace proj
