// Per-kernel CUDA-event tracing (projection_trace_enable / _read).
#include <mutex>
#include <string.h>
#include <string>
#include <vector>

#include "common.cuh"

namespace proj {
namespace {

struct Record {
    std::string name;
    cudaEvent_t ev[2];
};

std::mutex g_mu;
bool g_on = false;
std::vector<Record> g_rec;   // events are reused across enable() calls
size_t g_used = 0;

// inside a stream capture the record becomes an event-record node of the
// graph, so the pair still times the kernel when the graph runs
void record(cudaEvent_t ev, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, st);
}

}  // namespace

TraceSpan::TraceSpan(const char *name, cudaStream_t st) : st_(st) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return;
    if (g_used == g_rec.size()) {
        Record r;
        if (cudaEventCreate(&r.ev[0]) != cudaSuccess) return;
        if (cudaEventCreate(&r.ev[1]) != cudaSuccess) { cudaEventDestroy(r.ev[0]); return; }
        g_rec.push_back(r);
    }
    slot_ = (int)g_used++;
    g_rec[slot_].name = name;
    record(g_rec[slot_].ev[0], st_);
}

void TraceSpan::end() {
    if (slot_ < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    record(g_rec[slot_].ev[1], st_);
    slot_ = -1;
}

bool trace_active() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_on;
}

}  // namespace proj

using namespace proj;

extern "C" int projection_trace_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
    if (g_on) g_used = 0;
    return PROJ_OK;
}

extern "C" int projection_trace_read(const char *prefix, double *total_ms, int64_t *launches) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!total_ms || !launches) { set_error("NULL output"); return PROJ_EINVAL; }
    const size_t n = prefix ? strlen(prefix) : 0;
    double ms = 0.0;
    int64_t cnt = 0;
    for (size_t i = 0; i < g_used; ++i) {
        const Record &r = g_rec[i];
        if (n && r.name.compare(0, n, prefix) != 0) continue;
        cudaError_t e = cudaEventSynchronize(r.ev[1]);
        float f = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&f, r.ev[0], r.ev[1]);
        if (e != cudaSuccess) {
            set_error("trace event: %s", cudaGetErrorString(e));
            return PROJ_ECUDA;
        }
        ms += f;
        ++cnt;
    }
    *total_ms = ms;
    *launches = cnt;
    return PROJ_OK;
}
