// The C ABI of libmt (declared in include/mt.h): argument checks, workspace
// layout, status handling, and the launches of the device steps.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "../../include/mt.h"
#include "mt_device.cuh"
#include "mt_internal.h"

namespace mt {

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace layout (all offsets 256-byte aligned):
//   [0, 256)     status word, round flag
//   [256, 512)   meta: npairs, number of roots, root
//   [512, ...)   per-chunk counts of the ordered compaction
//   then, for a build, the face buffers (face_words(v) u32 per tile of the
//   tile shape v in use: 16^3, or 32x16x16 with MT_CFG_LARGE_TILES)
size_t workspace_bytes(uint64_t n)
{
    const uint64_t nchunks = (n + kCompactChunk - 1) / kCompactChunk;
    return 512 + align256(nchunks * sizeof(uint32_t));
}

size_t build_workspace_bytes(uint32_t nx, uint32_t ny, uint32_t nz)
{
    const uint64_t n = (uint64_t)nx * ny * nz;
    const uint64_t f0 = tile_count(0, nx, ny, nz) * face_words(0), f2 = tile_count(2, nx, ny, nz) * face_words(2);
    return workspace_bytes(n) + align256((f0 > f2 ? f0 : f2) * sizeof(uint32_t));
}

uint32_t *build_faces(void *base, uint64_t n)
{
    return reinterpret_cast<uint32_t *>(static_cast<char *>(base) + workspace_bytes(n));
}

bool carve_workspace(void *base, size_t bytes, uint64_t n, Workspace &ws)
{
    if (!base || ((uintptr_t)base & 255) || bytes < workspace_bytes(n)) return false;
    char *p = static_cast<char *>(base);
    ws.status = reinterpret_cast<uint32_t *>(p);
    ws.meta = reinterpret_cast<uint64_t *>(p + 256);
    ws.counts = reinterpret_cast<uint32_t *>(p + 512);
    ws.nchunks = (n + kCompactChunk - 1) / kCompactChunk;
    return true;
}

int device_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
    return sms;
}

// Checks a grid; returns MT_OK and n, or the error.
static mt_status grid_n(mt_grid g, uint64_t &n)
{
    if (g.nx == 0 || g.ny == 0 || g.nz == 0) return MT_ERR_INVALID;
    n = (uint64_t)g.nx * g.ny * g.nz;
    if (n >= 0xFFFFFFFFull) return MT_ERR_TOO_LARGE;
    return MT_OK;
}

// Small results (pair count, roots, status word) come back to the host
// through mapped pinned memory written by a one-thread kernel, not through a
// device-to-host copy: a copy would queue on the copy engine behind any large
// download another stream has in flight (such as the caller's copy of a
// previous field's triplets) and stall the call for its whole duration.
// One buffer per host thread, allocated on first use and kept.
__global__ void k_readback(const uint64_t *meta, const uint32_t *status, volatile uint64_t *out)
{
    if (meta) {
        out[0] = meta[0];
        out[1] = meta[1];
        out[2] = meta[2];
    }
    out[3] = *status;
}

// out[0..2] = meta (if given), out[3] = status word; synchronises s
cudaError_t readback(const uint64_t *meta, const uint32_t *status, cudaStream_t s, uint64_t out[4])
{
    thread_local uint64_t *h = nullptr, *d = nullptr;
    if (!h) {
        void *hp = nullptr, *dp = nullptr;
        cudaError_t e = cudaHostAlloc(&hp, 64, cudaHostAllocMapped | cudaHostAllocPortable);
        if (e != cudaSuccess) return e;
        if ((e = cudaHostGetDevicePointer(&dp, hp, 0)) != cudaSuccess) {
            cudaFreeHost(hp);
            return e;
        }
        h = static_cast<uint64_t *>(hp), d = static_cast<uint64_t *>(dp);
    }
    k_readback<<<1, 1, 0, s>>>(meta, status, d);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    const volatile uint64_t *vh = h;
    for (int i = 0; i < 4; i++) out[i] = vh[i];
    return cudaSuccess;
}

mt_status status_from_bits(uint32_t bits)
{
    if (bits & ST_NONFINITE) return MT_ERR_NONFINITE;
    if (bits & ST_TIMEOUT) return MT_ERR_TIMEOUT;
    if (bits & ST_CAPACITY) return MT_ERR_CAPACITY;
    if (bits & ST_CORRUPT) return MT_ERR_INVALID;
    return MT_OK;
}

}  // namespace mt

using namespace mt;

extern "C" {

const char *mt_status_str(mt_status st)
{
    switch (st) {
    case MT_OK: return "ok";
    case MT_ERR_INVALID: return "invalid argument";
    case MT_ERR_TOO_LARGE: return "grid too large (n >= 2^32 - 1)";
    case MT_ERR_NONFINITE: return "field holds a non-finite value";
    case MT_ERR_CAPACITY: return "output buffer too small";
    case MT_ERR_CUDA: return "CUDA runtime error";
    case MT_ERR_NOMEM: return "out of device memory";
    case MT_ERR_TIMEOUT: return "bounded device loop hit its limit";
    case MT_ERR_BUSY: return "not finished yet";
    default: return "unknown status";
    }
}

size_t mt_workspace_bytes(mt_grid g)
{
    uint64_t n;
    if (grid_n(g, n) != MT_OK) return 0;
    return build_workspace_bytes(g.nx, g.ny, g.nz);
}

mt_status mt_build_triplets_ex(const float *d_f, mt_grid g, uint64_t *d_W, void *d_ws, size_t ws_bytes, uint32_t flags,
                               void *stream)
{
    return mt_build_triplets_cfg(d_f, g, d_W, d_ws, ws_bytes, flags, 0u, stream);
}

mt_status mt_build_triplets_cfg(const float *d_f, mt_grid g, uint64_t *d_W, void *d_ws, size_t ws_bytes, uint32_t flags,
                                uint32_t cfg, void *stream)
{
    if (cfg & ~MT_CFG_SINGLE_MASK) return MT_ERR_INVALID;
    uint64_t n;
    mt_status st = grid_n(g, n);
    if (st != MT_OK) return st;
    if (!d_f || !d_W || ((uintptr_t)d_f & 3) || ((uintptr_t)d_W & 7) || (flags & ~MT_SUPERLEVEL))
        return MT_ERR_INVALID;
    Workspace ws;
    if (ws_bytes < build_workspace_bytes(g.nx, g.ny, g.nz) || !carve_workspace(d_ws, ws_bytes, n, ws))
        return MT_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(ws.status, 0, 256, s) != cudaSuccess) return MT_ERR_CUDA;
    const float sg = (flags & MT_SUPERLEVEL) ? -1.0f : 1.0f;
    if (launch_build(d_f, d_W, g.nx, g.ny, g.nz, ws, build_faces(d_ws, n), sg, s, cfg) != cudaSuccess)
        return MT_ERR_CUDA;
    return MT_OK;
}

mt_status mt_build_components(const float *d_f, mt_grid g, uint64_t *d_W, float t, float eps, uint32_t flags,
                              uint32_t cfg, uint32_t *d_labels, void *d_ws, size_t ws_bytes, void *stream)
{
    if (cfg & ~MT_CFG_SINGLE_MASK) return MT_ERR_INVALID;
    uint64_t n;
    mt_status st = grid_n(g, n);
    if (st != MT_OK) return st;
    if (!d_f || !d_W || !d_labels || std::isnan(t) || std::isnan(eps) || ((uintptr_t)d_f & 3) ||
        ((uintptr_t)d_W & 7) || ((uintptr_t)d_labels & 3) || (flags & ~MT_SUPERLEVEL))
        return MT_ERR_INVALID;
    Workspace ws;
    if (ws_bytes < build_workspace_bytes(g.nx, g.ny, g.nz) || !carve_workspace(d_ws, ws_bytes, n, ws))
        return MT_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(ws.status, 0, 256, s) != cudaSuccess) return MT_ERR_CUDA;
    const float sg = (flags & MT_SUPERLEVEL) ? -1.0f : 1.0f;
    const LabelArgs la{d_labels, sg * t, eps};
    if (launch_build(d_f, d_W, g.nx, g.ny, g.nz, ws, build_faces(d_ws, n), sg, s, cfg, &la) != cudaSuccess)
        return MT_ERR_CUDA;
    return MT_OK;
}

mt_status mt_build_step(const float *d_f, mt_grid g, uint64_t *d_W, float t, float eps, uint32_t flags, uint32_t cfg,
                        uint32_t *d_labels, uint32_t *d_pairs, uint64_t cap, uint64_t *h_npairs, uint32_t *h_root,
                        void *d_ws, size_t ws_bytes, void *stream)
{
    if (cfg & ~MT_CFG_SINGLE_MASK) return MT_ERR_INVALID;
    uint64_t n;
    mt_status st = grid_n(g, n);
    if (st != MT_OK) return st;
    if (!d_f || !d_W || !d_labels || !h_npairs || std::isnan(t) || std::isnan(eps) || ((uintptr_t)d_f & 3) ||
        ((uintptr_t)d_W & 7) || ((uintptr_t)d_labels & 3) || (cap && (!d_pairs || ((uintptr_t)d_pairs & 3))) ||
        (flags & ~MT_SUPERLEVEL))
        return MT_ERR_INVALID;
    Workspace ws;
    if (ws_bytes < build_workspace_bytes(g.nx, g.ny, g.nz) || !carve_workspace(d_ws, ws_bytes, n, ws))
        return MT_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(ws.status, 0, 256, s) != cudaSuccess) return MT_ERR_CUDA;
    const float sg = (flags & MT_SUPERLEVEL) ? -1.0f : 1.0f;
    const LabelArgs la{d_labels, sg * t, eps};
    if (launch_build(d_f, d_W, g.nx, g.ny, g.nz, ws, build_faces(d_ws, n), sg, s, cfg, &la) != cudaSuccess)
        return MT_ERR_CUDA;
    if (launch_pairs(d_W, n, d_pairs, cap, ws, s, d_f, sg, eps) != cudaSuccess) return MT_ERR_CUDA;
    uint64_t meta[4];
    if (readback(ws.meta, ws.status, s, meta) != cudaSuccess) return MT_ERR_CUDA;
    const uint32_t bits = (uint32_t)meta[3];
    if (bits) return status_from_bits(bits);
    *h_npairs = meta[0];
    if (h_root) *h_root = meta[1] == 1 ? (uint32_t)meta[2] : 0xFFFFFFFFu;
    if (meta[1] != 1) return MT_ERR_INVALID;  // not a tree of a connected grid
    return meta[0] > cap ? MT_ERR_CAPACITY : MT_OK;
}

mt_status mt_build_autotune(const float *d_f, mt_grid g, uint64_t *d_W, void *d_ws, size_t ws_bytes, uint32_t flags,
                            void *stream, float *ms, uint32_t *best)
{
    if (!ms || !best) return MT_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess) return MT_ERR_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return MT_ERR_CUDA;
    }
    constexpr int kCfgs = 8;  // the even configurations 0 .. 14
    mt_status st = MT_OK;
    for (int i = 0; i < kCfgs && st == MT_OK; i++) {
        const uint32_t cfg = 2u * (uint32_t)i;
        st = mt_build_triplets_cfg(d_f, g, d_W, d_ws, ws_bytes, flags, cfg, stream);  // warm-up
        float best_ms = 1e30f;
        for (int rep = 0; rep < 3 && st == MT_OK; rep++) {
            cudaEventRecord(a, s);
            st = mt_build_triplets_cfg(d_f, g, d_W, d_ws, ws_bytes, flags, cfg, stream);
            cudaEventRecord(b, s);
            if (cudaEventSynchronize(b) != cudaSuccess) st = MT_ERR_CUDA;
            float t = 0.f;
            cudaEventElapsedTime(&t, a, b);
            if (t < best_ms) best_ms = t;
        }
        ms[i] = best_ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != MT_OK) return st;
    int k = 0;
    for (int i = 1; i < kCfgs; i++)
        if (ms[i] < ms[k]) k = i;
    *best = 2u * (uint32_t)k;
    return mt_sync_status(d_ws, stream);
}

mt_status mt_build_triplets(const float *d_f, mt_grid g, uint64_t *d_W, void *d_ws, size_t ws_bytes, void *stream)
{
    return mt_build_triplets_ex(d_f, g, d_W, d_ws, ws_bytes, 0u, stream);
}

mt_status mt_persistence_pairs(const float *d_f, const uint64_t *d_W, mt_grid g, uint32_t *d_pairs, uint64_t cap,
                               uint64_t *h_npairs, uint32_t *h_root, void *d_ws, size_t ws_bytes, void *stream)
{
    uint64_t n;
    mt_status st = grid_n(g, n);
    if (st != MT_OK) return st;
    if (!d_f || !d_W || !h_npairs || ((uintptr_t)d_W & 7) || (cap && (!d_pairs || ((uintptr_t)d_pairs & 3))))
        return MT_ERR_INVALID;
    Workspace ws;
    if (!carve_workspace(d_ws, ws_bytes, n, ws)) return MT_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (launch_pairs(d_W, n, d_pairs, cap, ws, s) != cudaSuccess) return MT_ERR_CUDA;
    uint64_t meta[4];
    if (readback(ws.meta, ws.status, s, meta) != cudaSuccess) return MT_ERR_CUDA;
    const uint32_t bits = (uint32_t)meta[3];
    if (bits) return status_from_bits(bits);
    *h_npairs = meta[0];
    if (h_root) *h_root = meta[1] == 1 ? (uint32_t)meta[2] : 0xFFFFFFFFu;
    if (meta[1] != 1) return MT_ERR_INVALID;  // not a tree of a connected grid
    return meta[0] > cap ? MT_ERR_CAPACITY : MT_OK;
}

mt_status mt_simplified_pairs(const float *d_f, const uint64_t *d_W, mt_grid g, float eps, uint32_t flags,
                              uint32_t *d_pairs, uint64_t cap, uint64_t *h_npairs, uint32_t *h_root, void *d_ws,
                              size_t ws_bytes, void *stream)
{
    uint64_t n;
    mt_status st = grid_n(g, n);
    if (st != MT_OK) return st;
    if (!d_f || !d_W || !h_npairs || std::isnan(eps) || ((uintptr_t)d_f & 3) || ((uintptr_t)d_W & 7) ||
        (cap && (!d_pairs || ((uintptr_t)d_pairs & 3))) || (flags & ~MT_SUPERLEVEL))
        return MT_ERR_INVALID;
    Workspace ws;
    if (!carve_workspace(d_ws, ws_bytes, n, ws)) return MT_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float sg = (flags & MT_SUPERLEVEL) ? -1.0f : 1.0f;
    if (launch_pairs(d_W, n, d_pairs, cap, ws, s, d_f, sg, eps) != cudaSuccess) return MT_ERR_CUDA;
    uint64_t meta[4];
    if (readback(ws.meta, ws.status, s, meta) != cudaSuccess) return MT_ERR_CUDA;
    const uint32_t bits = (uint32_t)meta[3];
    if (bits) return status_from_bits(bits);
    *h_npairs = meta[0];
    if (h_root) *h_root = meta[1] == 1 ? (uint32_t)meta[2] : 0xFFFFFFFFu;
    if (meta[1] != 1) return MT_ERR_INVALID;  // not a tree of a connected grid
    return meta[0] > cap ? MT_ERR_CAPACITY : MT_OK;
}

mt_status mt_simplified_components_at(const float *d_f, const uint64_t *d_W, mt_grid g, float t, float eps,
                                      uint32_t flags, uint32_t *d_labels, void *d_ws, size_t ws_bytes, void *stream)
{
    uint64_t n;
    mt_status st = grid_n(g, n);
    if (st != MT_OK) return st;
    if (!d_f || !d_W || !d_labels || std::isnan(t) || std::isnan(eps) || ((uintptr_t)d_f & 3) ||
        ((uintptr_t)d_W & 7) || ((uintptr_t)d_labels & 3) || (flags & ~MT_SUPERLEVEL))
        return MT_ERR_INVALID;
    Workspace ws;
    if (!carve_workspace(d_ws, ws_bytes, n, ws)) return MT_ERR_INVALID;
    const float sg = (flags & MT_SUPERLEVEL) ? -1.0f : 1.0f;
    if (launch_labels(d_f, d_W, g.nx, g.ny, g.nz, sg * t, sg, d_labels, ws, static_cast<cudaStream_t>(stream), eps) !=
        cudaSuccess)
        return MT_ERR_CUDA;
    return MT_OK;
}

mt_status mt_components_at_ex(const float *d_f, const uint64_t *d_W, mt_grid g, float t, uint32_t flags,
                              uint32_t *d_labels, void *d_ws, size_t ws_bytes, void *stream)
{
    uint64_t n;
    mt_status st = grid_n(g, n);
    if (st != MT_OK) return st;
    if (!d_f || !d_W || !d_labels || std::isnan(t) || ((uintptr_t)d_W & 7) || ((uintptr_t)d_labels & 3) ||
        (flags & ~MT_SUPERLEVEL))
        return MT_ERR_INVALID;
    Workspace ws;
    if (!carve_workspace(d_ws, ws_bytes, n, ws)) return MT_ERR_INVALID;
    const float sg = (flags & MT_SUPERLEVEL) ? -1.0f : 1.0f;
    if (launch_labels(d_f, d_W, g.nx, g.ny, g.nz, sg * t, sg, d_labels, ws, static_cast<cudaStream_t>(stream)) !=
        cudaSuccess)
        return MT_ERR_CUDA;
    return MT_OK;
}

mt_status mt_components_at(const float *d_f, const uint64_t *d_W, mt_grid g, float t, uint32_t *d_labels,
                           void *d_ws, size_t ws_bytes, void *stream)
{
    return mt_components_at_ex(d_f, d_W, g, t, 0u, d_labels, d_ws, ws_bytes, stream);
}

mt_status mt_sync_status(void *d_ws, void *stream)
{
    if (!d_ws || ((uintptr_t)d_ws & 255)) return MT_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t rb[4];
    if (readback(nullptr, static_cast<const uint32_t *>(d_ws), s, rb) != cudaSuccess) return MT_ERR_CUDA;
    const uint32_t bits = (uint32_t)rb[3];
    if (bits && cudaMemsetAsync(d_ws, 0, sizeof(uint32_t), s) != cudaSuccess) return MT_ERR_CUDA;
    return status_from_bits(bits);
}

}  // extern "C"
