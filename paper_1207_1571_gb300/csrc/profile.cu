// profile.cu -- per-stage CUDA-event timing and launch counting.
//
// The paper times its solver components by instrumenting the host code
// around every kernel launch (Sec. 4.3.2); here each stage of a step is
// bracketed by two CUDA events on the mesh's stream, so the measured time is
// device time on the launching stream.  Recording is skipped while a stream
// is being captured into a graph.
#include <mutex>
#include <vector>

#include "fvgb_internal.h"

namespace fvgb {

namespace {
struct Rec {
    int stage;
    cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_pending;
std::vector<cudaEvent_t> g_pool;
double g_ms[FV_PROF_NSTAGE] = {};
long long g_launch[FV_PROF_NSTAGE] = {};

cudaEvent_t get_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

int prof_begin(int stage, cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return -1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return -1;
    Rec r{stage, get_event(), get_event()};
    if (!r.a || !r.b) return -1;
    cudaEventRecord(r.a, s);
    g_pending.push_back(r);
    return (int)g_pending.size() - 1;
}

void prof_end(int id, cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (id < 0 || id >= (int)g_pending.size()) return;
    cudaEventRecord(g_pending[id].b, s);
}

void prof_count(int stage, int n)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_launch[stage] += n;
}

}  // namespace fvgb

using namespace fvgb;

extern "C" fv_status fv_profile_enable(int32_t on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
    return FV_OK;
}

extern "C" fv_status fv_profile_read(double *ms, int64_t *launches, int32_t reset)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (Rec &r : g_pending) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_status(e, "cudaEventSynchronize");
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) g_ms[r.stage] += t;
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_pending.clear();
    for (int k = 0; k < FV_PROF_NSTAGE; ++k) {
        if (ms) ms[k] = g_ms[k];
        if (launches) launches[k] = g_launch[k];
        if (reset) { g_ms[k] = 0.0; g_launch[k] = 0; }
    }
    return FV_OK;
}
