// Host-side internals shared by the libmt translation units.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>

#include "../../include/mt.h"

namespace mt {

// Vertices per block of the ordered compactions (pairs): 256 threads x 16.
constexpr uint32_t kCompactChunk = 4096;

// One field as the kernels see it. In a batch, fields are packed one after
// another in the field, triplet and pair arenas, and tile0 / chunk0 number
// each field's first tile and first compaction chunk across the batch.
struct FieldDesc {
    const float *f;    // values, [nz][ny][nx]
    uint64_t *W;       // triplets, field-local vertex ids
    uint32_t *pairs;   // pair output ([cap][2]) or null
    uint64_t *meta;    // [0] npairs, [1] number of roots, [2] root
    uint32_t *faces;   // per tile: tile-local tops of the cross-edge ends, or null
    uint64_t n, cap;   // vertices, pair capacity
    uint64_t chunk0;   // first compaction chunk of the field
    uint32_t nx, ny, nz;
    uint32_t ntx, nty; // tiles along x and y for the tile shape in use
    uint32_t tile0;    // first tile of the field
    float sg = 1.0f;   // -1: the tree of -f (superlevel sets)
};

// Components of G_t read off the tree inside the repair pass of a build
// (mt_build_components): labels[u] as mt_simplified_components_at gives it.
struct LabelArgs {
    uint32_t *labels;  // uint32[n]
    float t;           // threshold on the values the order sees (sg * f)
    float eps;         // persistence simplification; <= 0: none
};

// Views into the caller's workspace (layout fixed by carve_workspace).
struct Workspace {
    uint32_t *status;  // status bits (ST_*)
    uint64_t *meta;    // [0] npairs, [1] number of roots, [2] root
    uint32_t *faces;   // per tile: tile-local tops of the cross-edge ends, or null vertex
    uint32_t *counts;  // per-chunk counts, then exclusive offsets in place
    uint64_t nchunks;
};

// Tracing (mt_trace.cu): phases timed with events on the launching stream.
enum Phase { kTile = 0, kMerge, kRepair, kPairs, kLabels, kBranches, kPhaseCount };
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

// The pair-compaction part of a workspace (status, counters, chunk counts)...
size_t workspace_bytes(uint64_t n);
bool carve_workspace(void *base, size_t bytes, uint64_t n, Workspace &ws);
// ...and the whole workspace a build needs: that part followed by the face
// buffers of k_tile / k_cross (build_faces points at them).
size_t build_workspace_bytes(uint32_t nx, uint32_t ny, uint32_t nz);
uint32_t *build_faces(void *base, uint64_t n);
// u32 entries of one tile's face buffer for tile variant v, and tile counts
uint32_t face_words(int variant);
uint64_t tile_count(int variant, uint32_t nx, uint32_t ny, uint32_t nz);
int device_sms();
// A kernel's function attributes (its dynamic shared-memory size, the
// carveout) belong to the context of one device, so a process that uses
// several GPUs sets them on each. One AttrFlags per kernel: pending() is true
// while the current device has not had them set (and always for device
// ordinals past the table), done() records that it has.
struct AttrFlags {
    static constexpr int kDevices = 64;
    std::atomic<bool> set[kDevices];
    bool pending(int &dev)
    {
        dev = -1;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) {
            dev = -1;
            return true;
        }
        return !set[dev].load(std::memory_order_relaxed);
    }
    void done(int dev)
    {
        if (dev >= 0) set[dev].store(true, std::memory_order_relaxed);
    }
};
// Reads meta[0..2] (if meta is given) and the status word into out[0..3]
// through mapped pinned memory (mt_api.cu); synchronises st.
cudaError_t readback(const uint64_t *meta, const uint32_t *status, cudaStream_t st, uint64_t out[4]);
mt_status status_from_bits(uint32_t bits);

// la: also label the components of G_t (null: triplets only)
cudaError_t launch_build(const float *f, uint64_t *W, uint32_t nx, uint32_t ny, uint32_t nz, Workspace &ws,
                         uint32_t *faces, float sg, cudaStream_t st, uint32_t cfg = 0,
                         const LabelArgs *la = nullptr);
// f, sg, eps: persistence simplification (pairs of persistence below eps
// dropped; eps <= 0 keeps all and does not read f)
cudaError_t launch_pairs(const uint64_t *W, uint64_t n, uint32_t *pairs, uint64_t cap, Workspace &ws,
                         cudaStream_t st, const float *f = nullptr, float sg = 1.0f, float eps = 0.0f);

// Batched build and pairs over a packed descriptor table already in device
// memory; cfg holds the MT_CFG_* knobs (mt_build.cu, mt_query.cu).
// The tile kernel for the wide-id path: in-tile merge tree of every
// 32x16x16 tile, written as 128-bit words of two 64-bit ids (mt_build.cu).
cudaError_t launch_tile_wide(const float *f, uint64_t *W2, uint32_t nx, uint32_t ny, uint32_t nz, float sg,
                             uint32_t *status, cudaStream_t st);
cudaError_t launch_batch_build(const FieldDesc *d_descs, uint32_t nfields, uint32_t ntiles, uint32_t cfg,
                               uint32_t *status, uint32_t *queue, cudaStream_t st);
cudaError_t launch_batch_pairs(const FieldDesc *d_descs, uint32_t nfields, uint64_t nchunks, uint32_t *counts,
                               uint64_t *npairs, const uint32_t *status, cudaStream_t st);
void tile_shape(int variant, uint32_t &tx, uint32_t &ty, uint32_t &tz);
cudaError_t launch_labels(const float *f, const uint64_t *W, uint32_t nx, uint32_t ny, uint32_t nz, float t,
                          float sg, uint32_t *labels, Workspace &ws, cudaStream_t st, float eps = 0.0f);

}  // namespace mt
