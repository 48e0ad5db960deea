// Batched triplet merge trees: many fields of uneven sizes, packed one after
// another in device arenas, built by one persistent tile kernel that takes
// tiles of every field from a device-side work queue, followed by one
// cross-tile merge, one repair and one pair compaction over all fields.
// mt_batch_prepare uploads the field table once; mt_batch_launch only
// enqueues memsets and kernels, so it can be captured in a CUDA graph and
// replayed.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "../../include/mt.h"
#include "mt_internal.h"

namespace mt {

mt_status status_from_bits(uint32_t bits);  // mt_api.cu

namespace {
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace of a batch (offsets 256-byte aligned):
//   [0, 256)    status word
//   [256, 512)  work-queue counter
//   descriptor tables for tile variants 0 and 1 (nfields each)
//   per-field meta (npairs, number of roots, root)
//   per-chunk counts of the pair compaction
//   face buffers of the tiles (sized for the larger of the two variants)
struct Layout {
    size_t descs[2], meta, counts, faces, total;
    uint32_t tiles[2];
    uint64_t chunks, vertices;
};

bool layout_of(const mt_grid *g, uint32_t nf, Layout &L)
{
    if (!g || nf == 0) return false;
    L.tiles[0] = L.tiles[1] = 0;
    L.chunks = L.vertices = 0;
    for (uint32_t i = 0; i < nf; i++) {
        if (g[i].nx == 0 || g[i].ny == 0 || g[i].nz == 0) return false;
        const uint64_t n = (uint64_t)g[i].nx * g[i].ny * g[i].nz;
        if (n >= 0xFFFFFFFFull) return false;
        for (int v = 0; v < 2; v++) {
            uint32_t tx, ty, tz;
            tile_shape(v, tx, ty, tz);
            const uint64_t t = (uint64_t)((g[i].nx + tx - 1) / tx) * ((g[i].ny + ty - 1) / ty) *
                               ((g[i].nz + tz - 1) / tz);
            if (L.tiles[v] + t >= 0x80000000ull) return false;
            L.tiles[v] += (uint32_t)t;
        }
        L.chunks += (n + kCompactChunk - 1) / kCompactChunk;
        L.vertices += n;
    }
    if (L.chunks >= 0x80000000ull) return false;
    size_t off = 512;
    for (int v = 0; v < 2; v++) {
        L.descs[v] = off;
        off = al256(off + (size_t)nf * sizeof(FieldDesc));
    }
    L.meta = off;
    off = al256(off + (size_t)nf * 3 * sizeof(uint64_t));
    L.counts = off;
    off = al256(off + (size_t)L.chunks * sizeof(uint32_t));
    L.faces = off;
    const uint64_t fw0 = (uint64_t)L.tiles[0] * face_words(0), fw1 = (uint64_t)L.tiles[1] * face_words(1);
    off = al256(off + (size_t)(fw0 > fw1 ? fw0 : fw1) * sizeof(uint32_t));
    L.total = off;
    return true;
}
}  // namespace

}  // namespace mt

using namespace mt;

extern "C" {

size_t mt_batch_workspace_bytes(const mt_grid *h_grids, uint32_t nfields)
{
    Layout L;
    return layout_of(h_grids, nfields, L) ? L.total : 0;
}

mt_status mt_batch_prepare(const float *d_arena, const mt_grid *h_grids, uint32_t nfields, uint64_t *d_W_arena,
                           uint32_t *d_pairs_arena, void *d_ws, size_t ws_bytes, mt_batch_plan *plan, void *stream)
{
    Layout L;
    if (!plan || !layout_of(h_grids, nfields, L)) return MT_ERR_INVALID;
    if (!d_arena || !d_W_arena || !d_pairs_arena || !d_ws || ((uintptr_t)d_ws & 255) || ws_bytes < L.total)
        return MT_ERR_INVALID;
    if (((uintptr_t)d_arena & 3) || ((uintptr_t)d_W_arena & 7) || ((uintptr_t)d_pairs_arena & 3))
        return MT_ERR_INVALID;
    char *ws = static_cast<char *>(d_ws);
    std::vector<FieldDesc> host(2 * (size_t)nfields);
    for (int v = 0; v < 2; v++) {
        uint32_t tx, ty, tz;
        tile_shape(v, tx, ty, tz);
        uint64_t off = 0, chunk0 = 0;
        uint32_t tile0 = 0;
        for (uint32_t i = 0; i < nfields; i++) {
            FieldDesc &d = host[(size_t)v * nfields + i];
            d = FieldDesc{};
            const mt_grid &g = h_grids[i];
            d.n = (uint64_t)g.nx * g.ny * g.nz;
            d.f = d_arena + off;
            d.W = d_W_arena + off;
            d.pairs = d_pairs_arena + 2 * off;
            d.meta = reinterpret_cast<uint64_t *>(ws + L.meta) + 3 * (size_t)i;
            d.cap = d.n;
            d.chunk0 = chunk0;
            d.nx = g.nx, d.ny = g.ny, d.nz = g.nz;
            d.ntx = (g.nx + tx - 1) / tx;
            d.nty = (g.ny + ty - 1) / ty;
            d.tile0 = tile0;
            d.faces = reinterpret_cast<uint32_t *>(ws + L.faces) + (size_t)tile0 * face_words(v);
            tile0 += d.ntx * d.nty * ((g.nz + tz - 1) / tz);
            chunk0 += (d.n + kCompactChunk - 1) / kCompactChunk;
            off += d.n;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int v = 0; v < 2; v++)
        if (cudaMemcpyAsync(ws + L.descs[v], host.data() + (size_t)v * nfields, (size_t)nfields * sizeof(FieldDesc),
                            cudaMemcpyHostToDevice, s) != cudaSuccess)
            return MT_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MT_ERR_CUDA;  // host table may go away after return
    plan->nfields = nfields;
    plan->tiles[0] = L.tiles[0];
    plan->tiles[1] = L.tiles[1];
    plan->chunks = L.chunks;
    plan->vertices = L.vertices;
    plan->ws_bytes = L.total;
    return MT_OK;
}

mt_status mt_batch_launch(const mt_batch_plan *plan, int cfg, uint64_t *d_npairs, void *d_ws, size_t ws_bytes,
                          void *stream)
{
    if (!plan || !d_npairs || !d_ws || ((uintptr_t)d_ws & 255) || ws_bytes < plan->ws_bytes || plan->nfields == 0 ||
        cfg < 0 || cfg >= MT_CFG_COUNT || ((uintptr_t)d_npairs & 7))
        return MT_ERR_INVALID;
    const int variant = (cfg & MT_CFG_SMALL_TILES) ? 1 : 0;
    Layout L;
    L.descs[0] = 512;
    L.descs[1] = al256(512 + (size_t)plan->nfields * sizeof(FieldDesc));
    L.meta = al256(L.descs[1] + (size_t)plan->nfields * sizeof(FieldDesc));
    L.counts = al256(L.meta + (size_t)plan->nfields * 3 * sizeof(uint64_t));
    char *ws = static_cast<char *>(d_ws);
    uint32_t *status = reinterpret_cast<uint32_t *>(ws);
    uint32_t *queue = reinterpret_cast<uint32_t *>(ws + 256);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(status, 0, 256, s) != cudaSuccess) return MT_ERR_CUDA;
    if (cudaMemsetAsync(ws + L.meta, 0, (size_t)plan->nfields * 3 * sizeof(uint64_t), s) != cudaSuccess)
        return MT_ERR_CUDA;
    const FieldDesc *descs = reinterpret_cast<const FieldDesc *>(ws + L.descs[variant]);
    if (launch_batch_build(descs, plan->nfields, plan->tiles[variant], (uint32_t)cfg, status, queue, s) != cudaSuccess)
        return MT_ERR_CUDA;
    if (launch_batch_pairs(descs, plan->nfields, plan->chunks, reinterpret_cast<uint32_t *>(ws + L.counts), d_npairs,
                           status, s) != cudaSuccess)
        return MT_ERR_CUDA;
    return MT_OK;
}

mt_status mt_batch_build(const float *d_arena, const mt_grid *h_grids, uint32_t nfields, uint64_t *d_W_arena,
                         uint32_t *d_pairs_arena, uint64_t *d_npairs, void *d_ws, size_t ws_bytes, void *stream)
{
    mt_batch_plan plan;
    mt_status st = mt_batch_prepare(d_arena, h_grids, nfields, d_W_arena, d_pairs_arena, d_ws, ws_bytes, &plan, stream);
    if (st != MT_OK) return st;
    return mt_batch_launch(&plan, 0, d_npairs, d_ws, ws_bytes, stream);
}

mt_status mt_batch_autotune(const mt_batch_plan *plan, uint64_t *d_npairs, void *d_ws, size_t ws_bytes, void *stream,
                            float *ms, int *best)
{
    if (!plan || !ms || !best) return MT_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess) return MT_ERR_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return MT_ERR_CUDA;
    }
    mt_status st = MT_OK;
    for (int c = 0; c < MT_CFG_COUNT && st == MT_OK; c++) {
        st = mt_batch_launch(plan, c, d_npairs, d_ws, ws_bytes, stream);  // warm-up
        if (st != MT_OK) break;
        float best_ms = 1e30f;
        for (int rep = 0; rep < 3 && st == MT_OK; rep++) {
            cudaEventRecord(a, s);
            st = mt_batch_launch(plan, c, d_npairs, d_ws, ws_bytes, stream);
            cudaEventRecord(b, s);
            if (cudaEventSynchronize(b) != cudaSuccess) st = MT_ERR_CUDA;
            float t = 0.f;
            cudaEventElapsedTime(&t, a, b);
            if (t < best_ms) best_ms = t;
        }
        ms[c] = best_ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != MT_OK) return st;
    int k = 0;
    for (int c = 1; c < MT_CFG_COUNT; c++)
        if (ms[c] < ms[k]) k = c;
    *best = k;
    uint32_t bits = 0;
    if (cudaMemcpy(&bits, d_ws, sizeof(bits), cudaMemcpyDeviceToHost) != cudaSuccess) return MT_ERR_CUDA;
    return status_from_bits(bits);
}

}  // extern "C"
