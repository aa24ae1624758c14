// Launch sequences replayed as CUDA graphs.  A body that only enqueues work
// (no allocation, no synchronisation) is captured on a private non-blocking
// stream and launched as one graph on the caller's stream.  The executable
// graph of each (device, slot) is kept per host thread and updated in place
// when the next capture has the same topology, so repeated searches of one
// shape pay neither re-instantiation nor per-kernel launch latency.
#include <stdlib.h>

#include <map>
#include <utility>

#include "common.cuh"

namespace proj {
namespace {

struct ThreadGraphs {
    std::map<int, cudaStream_t> capture_stream;                 // per device
    std::map<std::pair<int, int>, cudaGraphExec_t> exec;        // per (device, slot)
};
thread_local ThreadGraphs tl_graphs;

bool graphs_enabled() {
    static const bool on = [] {
        const char *e = getenv("PROJ_GRAPHS");
        return !(e && e[0] == '0');
    }();
    return on;
}

}  // namespace

int run_as_graph(int slot, cudaStream_t st, const std::function<int(cudaStream_t)> &body) {
    if (!graphs_enabled()) return body(st);
    int dev = 0;
    PROJ_CUDA_TRY(cudaGetDevice(&dev));
    cudaStream_t &cs = tl_graphs.capture_stream[dev];
    if (!cs) PROJ_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    PROJ_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const int rc = body(cs);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (rc != PROJ_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (rc != PROJ_OK) return rc;
        set_error("stream capture: %s", cudaGetErrorString(e));
        return PROJ_ECUDA;
    }
    cudaGraphExec_t &ex = tl_graphs.exec[{dev, slot}];
    // traced launches record their own events, which an update would not re-point
    if (ex && trace_active()) {
        cudaGraphExecDestroy(ex);
        ex = nullptr;
    }
    if (ex) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(ex, g, &info) != cudaSuccess) {
            (void)cudaGetLastError();
            cudaGraphExecDestroy(ex);
            ex = nullptr;
        }
    }
    cudaError_t ie = cudaSuccess;
    if (!ex) ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        ex = nullptr;
        set_error("cudaGraphInstantiate: %s", cudaGetErrorString(ie));
        return PROJ_ECUDA;
    }
    PROJ_CUDA_TRY(cudaGraphLaunch(ex, st));
    return PROJ_OK;
}

}  // namespace proj
