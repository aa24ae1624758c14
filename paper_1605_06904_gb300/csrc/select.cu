// Keeping only the largest enriched buckets (serving-scale searches refine the
// `top` buckets with the most member l-mers; equal sizes keep the (trial, key)
// order of the candidate list), and gathering their member lists into a
// compact CSR list for theta^0 and EM.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace proj {
namespace {

constexpr int kBins = 4096;  // bucket sizes >= kBins - 1 share the last bin

__global__ void size_hist_kernel(const int32_t *__restrict__ cnt, int64_t C,
                                 unsigned long long *__restrict__ bins) {
    __shared__ unsigned int h[kBins];
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) h[b] = 0u;
    __syncthreads();
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C;
         c += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[min(cnt[c], kBins - 1)], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < kBins; b += blockDim.x)
        if (h[b]) atomicAdd(&bins[b], (unsigned long long)h[b]);
}

// Candidates are split into contiguous ranges, one CTA each.  size_count_kernel
// counts, per range, the candidates larger than `cstar` and equal to it;
// size_select_kernel then walks its range in index order and keeps every
// candidate larger than `cstar` and the first `need_eq` of size `cstar` over
// the whole list (ballot scans keep the order): the position of a kept
// candidate is the number of larger ones before it plus min(number of
// size-cstar ones before it, need_eq), with the counts of earlier ranges added.
__global__ void __launch_bounds__(1024) size_count_kernel(const int32_t *__restrict__ cnt, int64_t C,
                                                          int cstar, int64_t per_block,
                                                          longlong2 *__restrict__ blk) {
    __shared__ long long s_a[32], s_b[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t lo = blockIdx.x * per_block, hi = min(C, lo + per_block);
    long long a = 0, b = 0;
    for (int64_t c = lo + tid; c < hi; c += 1024) {
        const int v = cnt[c];
        a += v > cstar;
        b += v == cstar;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) { s_a[warp] = a; s_b[warp] = b; }
    __syncthreads();
    if (tid == 0) {
        long long ta = 0, tb = 0;
        for (int w = 0; w < 32; ++w) { ta += s_a[w]; tb += s_b[w]; }
        blk[blockIdx.x] = make_longlong2(ta, tb);
    }
}

__global__ void __launch_bounds__(1024) size_select_kernel(const int32_t *__restrict__ cnt,
                                                           int64_t C, int cstar, int64_t need_eq,
                                                           int64_t per_block,
                                                           const longlong2 *__restrict__ blk,
                                                           int64_t *__restrict__ out_idx,
                                                           int32_t *__restrict__ out_cnt,
                                                           int64_t cap) {
    __shared__ int s_gt[33], s_eq[33];
    __shared__ long long s_base[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (warp == 0) {  // counts of the earlier ranges
        long long a = 0, b = 0;
        for (int q = lane; q < (int)blockIdx.x; q += 32) { a += blk[q].x; b += blk[q].y; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if (lane == 0) { s_base[0] = a; s_base[1] = b; }
    }
    __syncthreads();
    int64_t gt_seen = s_base[0], eq_seen = s_base[1];
    const int64_t lo = blockIdx.x * per_block, hi = min(C, lo + per_block);
    for (int64_t base = lo; base < hi; base += 1024) {
        const int64_t c = base + tid;
        const int v = c < hi ? cnt[c] : -1;
        const bool gt = v > cstar, eq = v == cstar;
        const unsigned bgt = __ballot_sync(0xffffffffu, gt), beq = __ballot_sync(0xffffffffu, eq);
        if (lane == 0) { s_gt[warp] = __popc(bgt); s_eq[warp] = __popc(beq); }
        __syncthreads();
        if (warp == 0) {
            int a = s_gt[lane], b = s_eq[lane];
            const int a0 = a, b0 = b;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int ua = __shfl_up_sync(0xffffffffu, a, o), ub = __shfl_up_sync(0xffffffffu, b, o);
                if (lane >= o) { a += ua; b += ub; }
            }
            s_gt[lane] = a - a0;  // exclusive prefix over warps
            s_eq[lane] = b - b0;
            if (lane == 31) { s_gt[32] = a; s_eq[32] = b; }
        }
        __syncthreads();
        const unsigned below = (1u << lane) - 1u;
        const int64_t gt_before = gt_seen + s_gt[warp] + __popc(bgt & below);
        const int64_t eq_before = eq_seen + s_eq[warp] + __popc(beq & below);
        if (gt || (eq && eq_before < need_eq)) {
            const int64_t pos = gt_before + (eq_before < need_eq ? eq_before : need_eq);
            if (pos < cap) {
                out_idx[pos] = c;
                out_cnt[pos] = v;
            }
        }
        gt_seen += s_gt[32];
        eq_seen += s_eq[32];
        __syncthreads();
    }
}

// Member lists of the selected candidates, copied into a compact CSR list.
__global__ void gather_members_kernel(const int64_t *__restrict__ sel, int64_t n,
                                      const int64_t *__restrict__ cand_off,
                                      const int32_t *__restrict__ members,
                                      const int64_t *__restrict__ new_off,
                                      int32_t *__restrict__ new_members) {
    const int64_t i = blockIdx.x;
    if (i >= n) return;
    const int64_t src = cand_off[sel[i]], len = new_off[i + 1] - new_off[i];
    for (int64_t e = threadIdx.x; e < len; e += blockDim.x) new_members[new_off[i] + e] = members[src + e];
}

}  // namespace

int select_top(const int32_t *cnt_dev, int64_t C, int64_t top, std::vector<int64_t> &sel,
               std::vector<int32_t> &sel_cnt, cudaStream_t st) {
    sel.clear();
    sel_cnt.clear();
    if (top <= 0 || C <= 0) return PROJ_OK;
    DevBuf bins, out;
    PROJ_TRY(bins.alloc(kBins * sizeof(unsigned long long), st));
    PROJ_CUDA_TRY(cudaMemsetAsync(bins.as<void>(), 0, kBins * sizeof(unsigned long long), st));
    const int grid = (int)std::min<int64_t>((C + 255) / 256, (int64_t)sm_count() * 4);
    {
        TraceSpan ts_("select", st);
        size_hist_kernel<<<grid, 256, 0, st>>>(cnt_dev, C, bins.as<unsigned long long>());
    }
    PROJ_LAUNCH_CHECK("size_hist_kernel");
    std::vector<unsigned long long> h(kBins);
    PROJ_CUDA_TRY(cudaMemcpyAsync(h.data(), bins.as<void>(), kBins * 8, cudaMemcpyDeviceToHost, st));
    PROJ_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t want = std::min(top, C);
    int cstar = 0;
    int64_t need_eq = 0, acc = 0;
    for (int b = kBins - 1; b >= 0; --b) {
        if (acc + (int64_t)h[b] >= want) {
            cstar = b;
            need_eq = want - acc;
            break;
        }
        acc += (int64_t)h[b];
    }
    if (cstar == kBins - 1) {
        // the threshold lies among saturated sizes: select on the host
        std::vector<int32_t> all(C);
        PROJ_CUDA_TRY(cudaMemcpyAsync(all.data(), cnt_dev, C * 4, cudaMemcpyDeviceToHost, st));
        PROJ_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<int64_t> idx(C);
        for (int64_t c = 0; c < C; ++c) idx[c] = c;
        std::stable_sort(idx.begin(), idx.end(),
                         [&](int64_t a, int64_t b) { return all[a] > all[b]; });
        idx.resize(want);
        sel = idx;
        for (int64_t c : sel) sel_cnt.push_back(all[c]);
        return PROJ_OK;
    }
    const int nblk = (int)std::min<int64_t>((C + 1023) / 1024, (int64_t)sm_count() * 2);
    const int64_t per_block = (C + nblk - 1) / nblk;
    PROJ_TRY(out.alloc(want * (sizeof(int64_t) + sizeof(int32_t)) + (size_t)nblk * sizeof(longlong2) + 16,
                       st));
    int64_t *oi = out.as<int64_t>();
    int32_t *oc = reinterpret_cast<int32_t *>(oi + want);
    longlong2 *blk = reinterpret_cast<longlong2 *>(
        (reinterpret_cast<uintptr_t>(oc + want) + 15) & ~(uintptr_t)15);
    {
        TraceSpan ts_("select", st);
        size_count_kernel<<<nblk, 1024, 0, st>>>(cnt_dev, C, cstar, per_block, blk);
    }
    PROJ_LAUNCH_CHECK("size_count_kernel");
    {
        TraceSpan ts_("select", st);
        size_select_kernel<<<nblk, 1024, 0, st>>>(cnt_dev, C, cstar, need_eq, per_block, blk, oi, oc,
                                                  want);
    }
    PROJ_LAUNCH_CHECK("size_select_kernel");
    std::vector<int64_t> picked(want);
    std::vector<int32_t> pc(want);
    PROJ_CUDA_TRY(cudaMemcpyAsync(picked.data(), oi, want * 8, cudaMemcpyDeviceToHost, st));
    PROJ_CUDA_TRY(cudaMemcpyAsync(pc.data(), oc, want * 4, cudaMemcpyDeviceToHost, st));
    PROJ_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int64_t> order(want);
    for (int64_t i = 0; i < want; ++i) order[i] = i;
    // picked is in index order; a stable sort by size keeps it for ties
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return pc[a] > pc[b]; });
    for (int64_t i : order) {
        sel.push_back(picked[i]);
        sel_cnt.push_back(pc[i]);
    }
    return PROJ_OK;
}

int gather_selected(const std::vector<int64_t> &sel, const std::vector<int32_t> &sel_cnt,
                    const int64_t *cand_off, const int32_t *members, DevBuf &out_buf,
                    int64_t **new_off, int32_t **new_members, cudaStream_t st) {
    const int64_t n = (int64_t)sel.size();
    std::vector<int64_t> off(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) off[i + 1] = off[i] + sel_cnt[i];
    PROJ_TRY(out_buf.alloc((size_t)(n + 1) * 8 + (size_t)n * 8 + (size_t)off[n] * 4 + 64, st));
    *new_off = out_buf.as<int64_t>();
    int64_t *sel_dev = *new_off + (n + 1);
    *new_members = reinterpret_cast<int32_t *>(sel_dev + n);
    PROJ_CUDA_TRY(cudaMemcpyAsync(*new_off, off.data(), (n + 1) * 8, cudaMemcpyHostToDevice, st));
    PROJ_CUDA_TRY(cudaMemcpyAsync(sel_dev, sel.data(), n * 8, cudaMemcpyHostToDevice, st));
    if (n > 0) {
        gather_members_kernel<<<(unsigned)n, 128, 0, st>>>(sel_dev, n, cand_off, members, *new_off,
                                                         *new_members);
        PROJ_LAUNCH_CHECK("gather_members_kernel");
    }
    return PROJ_OK;
}

}  // namespace proj
