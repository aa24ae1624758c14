// Instance and work-item descriptors of the tensor-core EM kernel, shared by
// the single-search and batched entry points.
#pragma once

#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace proj {

// One motif-search instance as the EM kernel sees it (device copy).
struct EmInst {
    const int32_t *seq_off;  // [t+1] positions of its sequences in the packed input
    const double *bg;        // [4] its background frequencies
    int t, l;
    int64_t cand_begin;      // index of its first candidate in the candidate arrays
    double gamma;            // site probability per sequence: < 1 ZOOPS, 1 OOPS
};

// One unit of EM work: up to 128 candidates of one instance against one
// contiguous range of that instance's sequences (group g of G).
struct EmItem {
    int64_t c0;      // first candidate (global index)
    int nc;          // candidates in this item (<= 128)
    int inst;        // instance index
    int seq_lo, seq_hi;
    int g;           // sequence group, selects the partial-result slot
    int n_tiles;     // tiles (64 or 128 l-mers) over the item's sequences
    int64_t tile0;   // index of its first tile in the run's one-hot tile array
};

// One sequence as the one-hot tile builder sees it.
struct XSeq {
    int64_t base;    // first base in the packed input
    int64_t tile;    // index of its first tile
    int ns, l;       // l-mers, motif length
};

// Host-side summary used to plan the items.
struct EmInstHost {
    int t = 0, l = 0;
    int64_t C = 0, cand_begin = 0;
    int64_t lmers = 0;
    const int32_t *seq_off = nullptr;  // host copy of the instance's EmInst::seq_off [t+1]
};

// h = parts per candidate row of the kernel (2: tiles of 64 l-mers, 4: 128)
int em_tc_plan(const std::vector<EmInstHost> &insts, std::vector<EmItem> &items, int &G,
               int ctas, int waves, int h);

// One tensor-core EM run split into allocation/planning (em_tc_prepare, may
// synchronise to autotune), launches only (em_tc_enqueue, capturable in a
// CUDA graph) and the error check (em_tc_finish, synchronises).
struct EmTcRun {
    const uint32_t *packed = nullptr;
    int64_t nwords = 0;
    const EmInst *inst_dev = nullptr;
    const float *theta0 = nullptr;
    int64_t C = 0;
    int stride = 0, n_inst = 0, kp = 16, G = 1, ctas = 3, n_items = 0, h = 2;
    DevBuf part, tmp, flag, items, tiles;
    DevBuf xt, xseq;  // one-hot tiles [n_x_tiles][32 h][kp] BF16 (K-major core layout), their sequences
};
int em_tc_prepare(const uint32_t *packed, int64_t nwords, const std::vector<EmInstHost> &insts,
                  const EmInst *inst_dev, const float *theta0, int64_t C, int stride,
                  EmTcRun &run, cudaStream_t st);
int em_tc_enqueue(EmTcRun &run, int iters, float beta, float *theta_out, double *ll,
                  cudaStream_t st);
// Checks the launches' timeout flag (synchronises), or with err_dev copies it
// there on the stream for the caller to check later.
int em_tc_finish(EmTcRun &run, cudaStream_t st, int *err_dev = nullptr);

// Runs iters EM iterations + a final E-step for the candidates of all
// instances (models theta0[C][stride], stride >= 4l of each instance).
int run_em_tc_batch(const uint32_t *packed, int64_t nwords, const std::vector<EmInstHost> &insts,
                    const EmInst *inst_dev, const float *theta0, int64_t C, int stride, int iters,
                    float beta, float *theta_out, double *ll, cudaStream_t st,
                    int *err_dev = nullptr);

}  // namespace proj
