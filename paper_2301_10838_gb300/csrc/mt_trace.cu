// Tracing: per-phase device time from CUDA events recorded on the launching
// stream around each step, and a count of the kernels libmt launched. Off by
// default; when off it costs one branch per step.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/mt.h"
#include "mt_internal.h"

namespace mt {

namespace {
struct Pending {
    int phase;
    cudaEvent_t a, b;
};
std::mutex g_mu;
std::atomic<int> g_on{0};
std::atomic<unsigned long long> g_launches{0};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;
double g_ms[kPhaseCount];
unsigned long long g_calls[kPhaseCount];

cudaEvent_t take_event()
{
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void drain_locked()
{
    for (auto &p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_ms[p.phase] += ms;
            g_calls[p.phase] += 1;
        }
        g_free.push_back(p.a);
        g_free.push_back(p.b);
    }
    g_pending.clear();
}
}  // namespace

const char *phase_name(int p)
{
    static const char *names[kPhaseCount] = {"tile", "merge", "repair", "pairs", "labels", "branches"};
    return (p >= 0 && p < kPhaseCount) ? names[p] : "?";
}

void count_launch(unsigned k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

PhaseScope::PhaseScope(int phase, cudaStream_t st) : phase_(phase), st_(st), a_(nullptr)
{
    if (!g_on.load(std::memory_order_relaxed)) return;
    // events recorded into a graph under capture would never be read back
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st_, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> g(g_mu);
    a_ = take_event();
    if (a_) cudaEventRecord(static_cast<cudaEvent_t>(a_), st_);
}

PhaseScope::~PhaseScope()
{
    if (!a_) return;
    std::lock_guard<std::mutex> g(g_mu);
    cudaEvent_t b = take_event();
    if (!b) return;
    cudaEventRecord(b, st_);
    g_pending.push_back({phase_, static_cast<cudaEvent_t>(a_), b});
}

}  // namespace mt

using namespace mt;

extern "C" {

void mt_trace_enable(int on)
{
    std::lock_guard<std::mutex> g(g_mu);
    g_on.store(on ? 1 : 0);
}

int mt_trace_read(mt_phase_time *out, int max_entries, int reset)
{
    std::lock_guard<std::mutex> g(g_mu);
    drain_locked();
    int k = 0;
    for (int p = 0; p < kPhaseCount; p++) {
        if (!g_calls[p]) continue;
        if (out && k < max_entries) {
            std::memset(&out[k], 0, sizeof(out[k]));
            std::strncpy(out[k].name, phase_name(p), sizeof(out[k].name) - 1);
            out[k].calls = g_calls[p];
            out[k].total_ms = g_ms[p];
        }
        k++;
    }
    if (reset) {
        std::memset(g_ms, 0, sizeof(g_ms));
        std::memset(g_calls, 0, sizeof(g_calls));
    }
    return k;
}

unsigned long long mt_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"
