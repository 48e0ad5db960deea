// Persistence pairs without any device allocation by the caller.
//
// Some callers of this library cannot obtain device memory for a workspace:
// a host application may reserve the whole GPU for its own memory pool and
// forbid any further cudaMalloc, or a latency-critical path may not afford the
// synchronisation and unpredictable latency that an allocation brings. For
// them mt_persistence_pairs_noalloc runs the same pair-compaction kernels as
// mt_persistence_pairs, but takes the scratch they need (status word, pair
// count, per-chunk counts) from one fixed array that is part of the library
// image itself. That array exists once on every GPU that loads the library
// and stays there until the process exits.
#include <cuda_runtime.h>

#include "../../include/mt.h"
#include "mt_internal.h"

namespace mt {

mt_status status_from_bits(uint32_t bits);  // mt_api.cu

// Largest grid the allocation-free call accepts (1024^3 vertices), and the
// scratch it needs: 512 bytes of status and counters plus one count per
// compaction chunk, about 1 MiB in all.
constexpr uint64_t kNoAllocMaxVertices = 1ull << 30;
constexpr uint64_t kNoAllocBytes = 512 + (kNoAllocMaxVertices / kCompactChunk) * sizeof(uint32_t);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
// Device address of the scratch array in the context current on the calling
// thread. In host code the symbol's name is only a host-side stand-in, so the
// address is looked up with cudaGetSymbolAddress. It is looked up on every
// call rather than cached: an address belongs to one context, and a caller
// may run in a context other than the device's primary one, or reset the
// device between calls. The lookup is a host-side query.
cudaError_t noalloc_scratch(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}
}  // namespace

}  // namespace mt

using namespace mt;

extern "C" mt_status mt_persistence_pairs_noalloc(const float *d_f, const uint64_t *d_W, mt_grid g,
                                                  uint32_t *d_pairs, uint64_t cap, uint64_t *h_npairs,
                                                  uint32_t *h_root, void *stream)
{
    if (g.nx == 0 || g.ny == 0 || g.nz == 0) return MT_ERR_INVALID;
    const uint64_t n = (uint64_t)g.nx * g.ny * g.nz;
    if (n > kNoAllocMaxVertices) return MT_ERR_TOO_LARGE;
    if (!d_f || !d_W || !h_npairs || ((uintptr_t)d_W & 7) || (cap && (!d_pairs || ((uintptr_t)d_pairs & 3))))
        return MT_ERR_INVALID;
    void *scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return MT_ERR_CUDA;
    Workspace ws;
    if (!carve_workspace(scratch, kNoAllocBytes, n, ws)) return MT_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the array keeps whatever the previous call left: start from a clear
    // status word (the pair counters are cleared by the pairs launch itself)
    if (cudaMemsetAsync(ws.status, 0, 256, s) != cudaSuccess) return MT_ERR_CUDA;
    if (launch_pairs(d_W, n, d_pairs, cap, ws, s) != cudaSuccess) return MT_ERR_CUDA;
    uint64_t meta[3] = {0, 0, 0};
    uint32_t bits = 0;
    if (cudaMemcpyAsync(meta, ws.meta, sizeof(meta), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MT_ERR_CUDA;
    if (cudaMemcpyAsync(&bits, ws.status, sizeof(bits), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return MT_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MT_ERR_CUDA;
    if (bits) return status_from_bits(bits);
    *h_npairs = meta[0];
    if (h_root) *h_root = meta[1] == 1 ? (uint32_t)meta[2] : 0xFFFFFFFFu;
    if (meta[1] != 1) return MT_ERR_INVALID;
    return meta[0] > cap ? MT_ERR_CAPACITY : MT_OK;
}
