// Host-side internals shared by the libmt translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace mt {

// Vertices per block of the ordered compactions (pairs): 256 threads x 16.
constexpr uint32_t kCompactChunk = 4096;

// Views into the caller's workspace (layout fixed by carve_workspace).
struct Workspace {
    uint32_t *status;  // status bits (ST_*)
    uint32_t *more;    // "another round needed" flag of iterative kernels
    uint64_t *meta;    // [0] npairs, [1] number of roots, [2] root vertex
    uint32_t *counts;  // per-chunk counts, then exclusive offsets in place
    uint64_t nchunks;
};

// Tracing (mt_trace.cu): phases timed with events on the launching stream.
enum Phase { kInit = 0, kDescend, kMerge, kRepair, kPairs, kLabels, kBatch, kTile, kPhaseCount };
const char *phase_name(int p);
void count_launch(unsigned k = 1);
class PhaseScope {
  public:
    PhaseScope(int phase, cudaStream_t st);
    ~PhaseScope();
    PhaseScope(const PhaseScope &) = delete;
    PhaseScope &operator=(const PhaseScope &) = delete;

  private:
    int phase_;
    cudaStream_t st_;
    void *a_;
};

size_t workspace_bytes(uint64_t n);
bool carve_workspace(void *base, size_t bytes, uint64_t n, Workspace &ws);
int device_sms();

cudaError_t launch_build(const float *f, uint64_t *W, uint32_t nx, uint32_t ny, uint32_t nz, Workspace &ws,
                         cudaStream_t st);
cudaError_t launch_pairs(const uint64_t *W, uint64_t n, uint32_t *pairs, uint64_t cap, Workspace &ws,
                         cudaStream_t st);
cudaError_t launch_labels(const float *f, const uint64_t *W, uint32_t nx, uint32_t ny, uint32_t nz, float t,
                          uint32_t *labels, Workspace &ws, cudaStream_t st);

}  // namespace mt
