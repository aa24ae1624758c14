// EM scoring and M-step contractions on the tcgen05 tensor cores (BF16 hi+lo
// split operands, FP32 accumulation in tensor memory).
#include "common.cuh"

namespace proj {

int run_em_tc(const uint32_t *, const Layout &, const double *, const float *, int64_t, int,
              float, float *, double *, cudaStream_t) {
    set_error("PROJ_EM_BF16_SPLIT is not available in this build");
    return PROJ_ENOTSUP;
}

}  // namespace proj
