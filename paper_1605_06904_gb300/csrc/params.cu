// Algorithm 2 step 1 ("if not specified") on the device for a batch of
// instances: k = l - d - 1, s = max(3, ceil(2x / 4^k)) (twice the mean bucket
// size, floored at the empirical 3), and m = ceil(log(1 - q) / log B) with
// B = P[Binomial(t, p) < s], p = C(l-d, k) / C(l, k), the trial count that
// finds the planted bucket with probability q (Section 5).  Serving pipelines
// that hold instance sizes on the device derive the parameters there.
#include <math.h>

#include "common.cuh"

namespace proj {
namespace {

__device__ double log_binom_d(int n, int r) {
    return lgamma((double)n + 1.0) - lgamma((double)r + 1.0) - lgamma((double)(n - r) + 1.0);
}

// One thread per instance.  A value already > 0 in k, s or m is kept; status
// per instance: 0 OK, -1 invalid, -2 no finite trial count (k > l - d) or a
// count above 2^24.
__global__ void params_kernel(int n, const int32_t *__restrict__ t, const int64_t *__restrict__ x,
                              const int32_t *__restrict__ l, const int32_t *__restrict__ d,
                              int32_t *__restrict__ k, int32_t *__restrict__ s,
                              int32_t *__restrict__ m, int32_t *__restrict__ status, double q) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ti = t[i], li = l[i], di = d[i];
    int ki = k[i], si = s[i], mi = m[i];
    if (ti < 1 || li < 1 || li > 32 || di < 0 || di >= li || x[i] < 0) {
        status[i] = -1;
        return;
    }
    if (ki == 0) ki = li - di - 1;
    if (ki < 1 || ki > li) {
        status[i] = -1;
        return;
    }
    if (si == 0) si = (int)fmax(3.0, ceil(2.0 * (double)x[i] / pow(4.0, (double)ki)));
    int st = 0;
    if (mi == 0) {
        if (ki > li - di || si < 1) {
            st = -2;
        } else {
            const double lp = log_binom_d(li - di, ki) - log_binom_d(li, ki);
            const double p = exp(lp);
            double below = 0.0;
            for (int c = 0; c < si && c <= ti; ++c)
                below += exp(log_binom_d(ti, c) + c * lp + (ti - c) * log1p(-p));
            if (below >= 1.0) st = -2;
            else if (below <= 0.0) mi = 1;
            else {
                const double mm = ceil(log(1.0 - q) / log(below));
                if (mm > (double)(1 << 24)) st = -2;
                else mi = (int)mm;
            }
        }
    }
    k[i] = ki;
    s[i] = si;
    m[i] = st == 0 ? mi : 0;
    status[i] = st;
}

}  // namespace
}  // namespace proj

using namespace proj;

extern "C" int projection_params_batch(int n, const int32_t *t_dev, const int64_t *x_dev,
                                       const int32_t *l_dev, const int32_t *d_dev, int32_t *k_dev,
                                       int32_t *s_dev, int32_t *m_dev, int32_t *status_dev,
                                       double q, void *stream) {
    clear_error();
    PROJ_REQUIRE(n >= 0, "n must be >= 0");
    PROJ_REQUIRE(q > 0.0 && q < 1.0, "need 0 < q < 1");
    if (n == 0) return PROJ_OK;
    PROJ_REQUIRE(t_dev && x_dev && l_dev && d_dev && k_dev && s_dev && m_dev && status_dev,
                 "NULL device array");
    cudaStream_t st = (cudaStream_t)stream;
    {
        TraceSpan ts_("params", st);
        params_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, t_dev, x_dev, l_dev, d_dev, k_dev, s_dev,
                                                       m_dev, status_dev, q);
    }
    PROJ_LAUNCH_CHECK("params_kernel");
    return PROJ_OK;
}
